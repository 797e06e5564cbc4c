"""The tiled schedule with the dealt relabeling (the default): GPU against
the oracle run on the relabeled instance, results exchanged in caller
labels."""
import numpy as np
import pytest

from instances import planted_partition, chung_lu, workload
from relabel import RelabeledOracle

pytestmark = pytest.mark.gpu


def _solver(n, d, w, **kw):
    import paper_1901_10084_gb300 as cc
    return cc.Solver(n, d, w, interleave=True, **kw)


def _state(s):
    x, f = s.get_x()
    yt, yp = s.get_duals()
    return x, f, yt, yp


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0))


@pytest.mark.parametrize("n,tile,weighted", [(60, 16, False), (61, 8, True), (100, 16, True), (37, 32, False)])
def test_interleaved_exact_is_bitwise_equal(n, tile, weighted):
    d, w, _ = planted_partition(n, 4, 0.8, 0.1, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = RelabeledOracle(n, d, w, 0.2, tile)
    with _solver(n, d, w, tile=tile, exact=True) as s:
        for k in (1, 2):
            s.sweep(k)
            o.sweep(k)
            x, f, yt, yp = _state(s)
            np.testing.assert_array_equal(x, o.x)
            np.testing.assert_array_equal(f, o.f)
            np.testing.assert_array_equal(yt, o.ytri)
            np.testing.assert_array_equal(yp, o.ypair)
        assert s.check()["max_violation"] == o.max_violation()


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("n,tile,weighted", [(120, 16, False), (90, 8, True)])
def test_interleaved_fused_one_sweep(n, tile, weighted, precision):
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = RelabeledOracle(n, d, w, 0.2, tile)
    o.sweep(3)
    tol = 1e-12 if precision == "fp64" else 1e-5
    with _solver(n, d, w, tile=tile, precision=precision) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        s.sweep(1)
        o.sweep(1)
        x, f, yt, yp = _state(s)
        assert _rel(x, o.x) <= tol and _rel(f, o.f) <= tol
        assert _rel(yt, o.ytri) <= tol and _rel(yp, o.ypair) <= tol


def test_interleaved_converges_like_the_oracle():
    n, d, w, _ = workload("planted60")
    o = RelabeledOracle(n, d, w, 0.2, 16)
    ko = o.st.solve(1e-4, 5000, schedule=2, tile=16, check_every=1)
    with _solver(n, d, w, tile=16, check_every=1) as s:
        conv, kg = s.solve(1e-4, 5000)
        st = s.check()
    assert conv and kg == ko
    assert abs(st["lp_objective"] - o.objectives()["lp"]) <= 1e-6 * o.objectives()["lp"]


def test_interleaved_warm_start_and_resync():
    n = 80
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=8, weights=(0.5, 2.0))
    o = RelabeledOracle(n, d, w, 0.2, 16)
    o.sweep(4)
    with _solver(n, d, w, tile=16) as s:
        s.set_duals(o.ytri, o.ypair)
        x, f = s.get_x()
        assert _rel(x, o.x) <= 1e-12 and _rel(f, o.f) <= 1e-12
