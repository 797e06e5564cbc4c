"""l2 metric nearness on the GPU (problem="l2": min sum w (x - d)^2 over the
metric rows, Eq. metricnear with p = 2, solved as Eq. qp with eps = 1 and
c = -W d) against the oracle's l2 mode, through the C ABI.  Same bars as the
CC tests: exact mode bit for bit, fused form 1e-12 per sweep from an
identical state, the objective at convergence 1e-6 relative."""
import itertools

import numpy as np
import pytest

import oracle
from instances import noisy_euclidean, random_dissimilarity

pytestmark = pytest.mark.gpu

TOL_SWEEP = 1e-12


def _solver(n, d, w, **kw):
    import paper_1901_10084_gb300 as cc
    kw.setdefault("interleave", False)
    return cc.Solver(n, d, w, problem="l2", **kw)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0)) if a.size else 0.0


def _inputs(kind, n, seed, weighted):
    if kind == "rand":
        return random_dissimilarity(n, seed, weights=(0.5, 2.0) if weighted else None)
    d, w = noisy_euclidean(n, 2, 0.3, seed)
    if weighted:
        w = np.random.default_rng(seed + 7).uniform(0.5, 2.0, len(d))
    return d, w


@pytest.mark.parametrize("schedule,tile", [(2, 8), (2, 16), (1, 16), (0, 16)])
@pytest.mark.parametrize("n,kind,weighted", [(40, "rand", False), (45, "euc", True), (17, "rand", True)])
def test_exact_mode_is_bitwise_equal(schedule, tile, n, kind, weighted):
    d, w = _inputs(kind, n, n, weighted)
    o = oracle.State(n, d, w, problem="l2")
    with _solver(n, d, w, schedule=schedule, tile=tile, exact=True) as s:
        for k in (1, 2):
            for _ in range(k):
                o.sweep(schedule, tile)
            s.sweep(k)
            x, f = s.get_x()
            yt, yp = s.get_duals()
            np.testing.assert_array_equal(x, o.x)
            np.testing.assert_array_equal(yt, o.ytri)
            assert not f.any() and not yp.any()
        assert s.check()["max_violation"] == o.max_violation()


@pytest.mark.parametrize("variant", [0, 1, 2, 4])
@pytest.mark.parametrize("n,tile,kind,weighted,pre", [(60, 16, "rand", False, 2), (61, 16, "euc", True, 3),
                                                      (150, 8, "rand", True, 1), (97, 32, "euc", False, 4)])
def test_fused_one_sweep_from_identical_state(variant, n, tile, kind, weighted, pre):
    if variant == 2 and tile > 16:
        pytest.skip("one warp per block triple needs tile <= 16")
    d, w = _inputs(kind, n, n + 1, weighted)
    o = oracle.State(n, d, w, problem="l2")
    for _ in range(pre):
        o.sweep(2, tile)
    with _solver(n, d, w, tile=tile, variant=variant) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        s.sweep(1)
        o.sweep(2, tile)
        x, _ = s.get_x()
        yt, _ = s.get_duals()
        assert _rel(x, o.x) <= TOL_SWEEP and _rel(yt, o.ytri) <= TOL_SWEEP


@pytest.mark.parametrize("schedule", [0, 1])
def test_paper_schedules_fused(schedule):
    n = 70
    d, w = _inputs("rand", n, 3, True)
    o = oracle.State(n, d, w, problem="l2")
    with _solver(n, d, w, schedule=schedule) as s:
        for _ in range(3):
            s.sweep(1)
            o.sweep(schedule)
            x, _ = s.get_x()
            assert _rel(x, o.x) <= 10 * TOL_SWEEP


def test_check_quantities_match_oracle():
    n = 80
    d, w = _inputs("euc", n, 5, True)
    o = oracle.State(n, d, w, problem="l2")
    with _solver(n, d, w, tile=16) as s:
        for _ in range(3):
            s.sweep(1)
            o.sweep(2, 16)
        st = s.check()
    ob = o.objectives()
    assert st["max_violation"] == pytest.approx(o.max_violation(), rel=1e-9, abs=1e-15)
    for k_gpu, k_ora in (("lp_objective", "lp"), ("qp_primal", "qp_primal"), ("dual_objective", "dual")):
        assert st[k_gpu] == pytest.approx(ob[k_ora], rel=1e-10, abs=1e-13)
    assert st["gap"] == pytest.approx(ob["gap"], rel=1e-8, abs=1e-12)
    assert st["pair_violation"] == 0.0 and st["wf"] == 0.0


@pytest.mark.parametrize("interleave", [False, True])
def test_converged_objective_matches_oracle(interleave):
    """Noisy Euclidean input (converges in a few hundred sweeps): solve to
    violation 1e-9 with the gap closed to 1e-9 relative on both sides."""
    n = 60
    d, w = _inputs("euc", n, 11, True)
    o = oracle.State(n, d, w, problem="l2")
    for _ in range(20000):
        o.sweep(2, 16)
        ob = o.objectives()
        if o.max_violation() <= 1e-9 and abs(ob["gap"]) <= 1e-9 * ob["qp_primal"]:
            break
    with _solver(n, d, w, tile=16, interleave=interleave, check_every=5) as s:
        conv, k = s.solve(1e-9, 20000)
        st = s.check()
        x, _ = s.get_x()
    assert conv and st["max_violation"] <= 1e-9 and abs(st["gap"]) <= 1e-9 * st["qp_primal"]
    assert st["lp_objective"] == pytest.approx(o.objectives()["lp"], rel=1e-6)
    assert np.max(np.abs(x - o.x)) <= 1e-5


def test_many_sweeps_track_the_oracle_on_random_dissimilarities():
    """U[0,1] dissimilarities keep many rows active for thousands of sweeps
    (Dykstra's slow regime); 300 sweeps of GPU and oracle stay together."""
    n = 50
    d, w = _inputs("rand", n, 13, True)
    o = oracle.State(n, d, w, problem="l2")
    with _solver(n, d, w, tile=8) as s:
        s.sweep(300)
        for _ in range(300):
            o.sweep(2, 8)
        x, _ = s.get_x()
        st = s.check()
    assert _rel(x, o.x) <= 1e-9
    assert st["lp_objective"] == pytest.approx(o.objectives()["lp"], rel=1e-9)


def test_metric_input_is_returned_unchanged():
    rng = np.random.default_rng(2)
    n = 90
    labels = rng.integers(0, 5, n)
    d = np.array([0.0 if labels[i] == labels[j] else 1.0 for i, j in itertools.combinations(range(n), 2)])
    w = rng.uniform(0.5, 2.0, len(d))
    with _solver(n, d, w, tile=16, interleave=True) as s:
        conv, k = s.solve(0.0, 50)
        x, f = s.get_x()
        yt, _ = s.get_duals()
        st = s.check()
    assert conv and k == 10
    assert np.array_equal(x, d) and not yt.any() and not f.any()
    assert st["lp_objective"] == 0.0 and st["gap"] == 0.0


def test_unsupported_combinations_are_refused():
    import paper_1901_10084_gb300 as cc
    from paper_1901_10084_gb300 import warmstart
    n = 30
    d, w = random_dissimilarity(n, 1)
    with pytest.raises(cc.CCError) as e:
        _solver(n, d, w, precision="fp32_refine")
    assert e.value.code == cc.CC_ERR_UNSUPPORTED
    with _solver(n, d, w, tile=8) as s:
        yt, yp = s.get_duals()
        with pytest.raises(cc.CCError) as e:
            s.set_duals(yt, yp)
        assert e.value.code == cc.CC_ERR_UNSUPPORTED
        with pytest.raises(cc.CCError) as e:
            s.warm_start(warmstart.init_params(0))
        assert e.value.code == cc.CC_ERR_UNSUPPORTED


@pytest.mark.parametrize("exact", [True, False])
def test_worked_triangle_case_on_gpu(exact):
    """Sec. II-B's worked projection (tests/golden/worked_triangle.json) as an
    l2 sweep of n = 3 through the C ABI."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_triangle.json")))
    for case in g["cases"]:
        d = np.array(case["x_before"])
        with _solver(3, d, np.ones(3), tile=8, exact=exact) as s:
            s.sweep(1)
            x, _ = s.get_x()
        np.testing.assert_allclose(x, case["x_after"], rtol=0, atol=4e-16)
