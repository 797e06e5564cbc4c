"""Batched form: many instances of uneven size in one launch per sweep.  Each
instance must evolve exactly as the oracle on that instance (relabeled
tiled schedule), and a batch solve must give each instance the solution of
its own solve."""
import numpy as np
import pytest

from instances import batch_planted, planted_partition
from relabel import RelabeledOracle

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0))


def _instances():
    out = batch_planted(7, 3, 70, 2, 5, 0.7, 0.05, seed=11)
    n, d, w = out[2]
    out[2] = (n, d, np.random.default_rng(0).uniform(0.5, 2.0, d.shape))   # one weighted instance
    return out


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_batch_sweeps_match_the_oracle_per_instance(tile, order):
    import paper_1901_10084_gb300 as cc
    inst = _instances()
    oracles = [RelabeledOracle(n, d, w, 0.2, tile) for n, d, w in inst]
    with cc.Batch(inst, tile=tile, batch_order=order) as b:
        b.sweep(3)
        for (n, d, w), o in zip(inst, oracles):
            o.sweep(3)
        for i, o in enumerate(oracles):
            s = b.instance(i)
            x, f = s.get_x()
            yt, yp = s.get_duals()
            assert _rel(x, o.x) <= 1e-12 and _rel(f, o.f) <= 1e-12
            assert _rel(yt, o.ytri) <= 1e-12 and _rel(yp, o.ypair) <= 1e-12
            assert s.stats()["sweeps"] == 3


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_batch_solve_matches_single_solves(precision):
    import paper_1901_10084_gb300 as cc
    inst = batch_planted(9, 20, 120, 2, 6, 0.7, 0.05, seed=5)
    with cc.Batch(inst, tile=16, precision=precision, check_every=5) as b:
        conv, _, per = b.solve(1e-6, 5000)
        assert conv and min(per) > 0
        for i, (n, d, w) in enumerate(inst):
            s = b.instance(i)
            st = s.check()
            assert st["max_violation"] <= 1e-6 and st["state_fp32"] == 0
            with cc.Solver(n, d, w, tile=16, precision=precision, check_every=5) as one:
                ok, k = one.solve(1e-6, 5000)
                assert ok and k == per[i]
                x1, _ = one.get_x()
            x, _ = s.get_x()
            if precision == "fp64":
                assert _rel(x, x1) <= 1e-12      # same order, same arithmetic
            else:
                assert np.max(np.abs(x - x1)) <= 1e-4
                assert 0 < st["fp32_sweeps"] <= per[i] - 5   # refinement sweeps ran in FP64


def test_autotuner_returns_a_valid_choice():
    import paper_1901_10084_gb300 as cc
    inst = batch_planted(6, 30, 90, 2, 5, 0.7, 0.05, seed=2)
    opts, ms = cc.autotune_batch(inst, trial_sweeps=2)
    assert opts["tile"] in (8, 16, 32) and opts["batch_order"] in (0, 1) and opts["variant"] in (0, 1) and ms > 0
    with cc.Batch(inst, **opts) as b:
        conv, _, _ = b.solve(1e-4, 3000)
        assert conv


def test_full_size_batch_of_256():
    """The batched configuration at full size (256 planted instances,
    n ~ U[50, 400], k ~ U[2, 8], p 0.7 / 0.05, seed 3): five batch sweeps give
    every sampled instance exactly its own handle's iterates."""
    import paper_1901_10084_gb300 as cc
    from instances import batch_planted
    inst = batch_planted(256, 50, 400, 2, 8, 0.7, 0.05, seed=3)
    with cc.Batch(inst, tile=16) as b:
        b.sweep(5)
        for i in range(0, 256, 37):
            n, d, w = inst[i]
            with cc.Solver(n, d, w, tile=16) as s:
                s.sweep(5)
                xs, fs = s.get_x()
                ys, _ = s.get_duals()
            x, f = b.instance(i).get_x()
            y, _ = b.instance(i).get_duals()
            assert np.array_equal(x, xs) and np.array_equal(f, fs) and np.array_equal(y, ys)
