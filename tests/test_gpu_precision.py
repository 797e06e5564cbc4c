"""FP32 bulk sweeps + FP64 refinement, the resync x = x0 - W^-1 A^T y/eps,
and warm starts from duals (GPU, through the C ABI)."""
import numpy as np
import pytest

import oracle
from instances import planted_partition, chung_lu, workload

pytestmark = pytest.mark.gpu


def _solver(n, d, w, **kw):
    """Tiled schedule on consecutive blocks (no relabeling), the order the
    oracle's schedule 2 walks; the relabeled order is tested separately."""
    import paper_1901_10084_gb300 as cc
    kw.setdefault("interleave", False)
    return cc.Solver(n, d, w, **kw)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0))


@pytest.mark.parametrize("n,tile,weighted", [(60, 16, False), (90, 8, True), (130, 32, True)])
def test_resync_rebuilds_x_and_f_from_the_duals(n, tile, weighted):
    """After FP64 sweeps, setting the same duals back rebuilds x and f from
    the invariant; they must equal the swept x and f up to rounding."""
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    with _solver(n, d, w, tile=tile) as s:
        s.sweep(7)
        x, f = s.get_x()
        yt, yp = s.get_duals()
        s.set_duals(yt, yp)
        x2, f2 = s.get_x()
    assert _rel(x2, x) <= 1e-12 and _rel(f2, f) <= 1e-12


def test_warm_start_from_oracle_duals_matches_oracle_state():
    n = 70
    d, w, _ = planted_partition(n, 3, 0.7, 0.2, seed=3, weights=(0.5, 2.0))
    o = oracle.State(n, d, w, 0.2)
    for _ in range(5):
        o.sweep(2, 16)
    with _solver(n, d, w, tile=16) as s:
        s.set_duals(o.ytri, o.ypair)
        x, f = s.get_x()
        assert _rel(x, o.x) <= 1e-12 and _rel(f, o.f) <= 1e-12
        s.sweep(1)
        o.sweep(2, 16)
        x, f = s.get_x()
        assert _rel(x, o.x) <= 1e-12 and _rel(f, o.f) <= 1e-12


@pytest.mark.parametrize("n,weighted", [(60, False), (150, True)])
def test_fp32_sweep_tracks_the_oracle_to_float_precision(n, weighted):
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    with _solver(n, d, w, tile=16, precision="fp32_refine") as s:
        for _ in range(3):
            o.sweep(2, 16)
        s.sweep(3)
        x, f = s.get_x()
        st = s.check()
    assert st["state_fp32"] == 1 and st["fp32_sweeps"] == 3
    assert _rel(x, o.x) <= 1e-5 and _rel(f, o.f) <= 1e-5


@pytest.mark.parametrize("name,tile", [("planted60", 16), ("chunglu300", 8)])
def test_fp32_refine_reaches_the_fp64_solution(name, tile):
    """Both forms solved to 1e-8: the LP objectives agree to 1e-6 relative
    (the QP optimum is unique) and the refined state is FP64."""
    n, d, w, _ = workload(name)
    with _solver(n, d, w, tile=tile, check_every=5) as a:
        conv_a, ka = a.solve(1e-8, 20000)
        sa = a.check()
        xa, _ = a.get_x()
    with _solver(n, d, w, tile=tile, check_every=5, precision="fp32_refine") as b:
        conv_b, kb = b.solve(1e-8, 20000)
        sb = b.check()
        xb, _ = b.get_x()
    assert conv_a and conv_b
    assert sb["state_fp32"] == 0 and 0 < sb["fp32_sweeps"] < kb
    assert sb["max_violation"] <= 1e-8
    assert abs(sb["lp_objective"] - sa["lp_objective"]) <= 1e-6 * abs(sa["lp_objective"])
    assert np.max(np.abs(xb - xa)) <= 1e-5


@pytest.mark.parametrize("name,check_every", [("chunglu1000", 10), ("chunglu1000", 5), ("chunglu300", 10)])
def test_fp32_refine_meets_the_fp64_objective_at_the_solve_tolerance(name, check_every):
    """The precision form's target at the tolerance the solve is run to
    (violation 1e-4): the FP32 bulk sweeps end at that tolerance, the
    refinement then runs opts.refine_sweeps (5) FP64 sweeps from x and f
    rebuilt out of the converted duals, and the LP objective of the result is
    within 1e-6 relative of the plain FP64 solve's; the violation meets the
    tolerance in FP64."""
    n, d, w, _ = workload(name)
    res = {}
    for prec in ("fp64", "fp32_refine"):
        with _solver(n, d, w, tile=16, precision=prec, check_every=check_every, interleave=True) as s:
            conv, k = s.solve(1e-4, 3000)
            st = s.check()
            res[prec] = (conv, k, st, s.get_x()[0])
    conv64, k64, s64, x64 = res["fp64"]
    conv32, k32, s32, x32 = res["fp32_refine"]
    assert conv64 and conv32
    assert s32["state_fp32"] == 0 and s32["max_violation"] <= 1e-4
    assert 0 < s32["fp32_sweeps"] and k32 - s32["fp32_sweeps"] >= 5
    assert abs(s32["lp_objective"] - s64["lp_objective"]) <= 1e-6 * abs(s64["lp_objective"])
    assert np.max(np.abs(x32 - x64)) <= 1e-3


def test_refinement_sweeps_follow_an_explicit_switch():
    """After cc_refine_fp64 the solve runs refine_sweeps FP64 sweeps before the
    tolerance may end it, even when the rebuilt state already meets it."""
    n, d, w, _ = workload("planted60")
    with _solver(n, d, w, tile=16, precision="fp32_refine", check_every=1, refine_sweeps=3) as s:
        s.sweep(200)
        s.refine_fp64()
        assert s.check()["max_violation"] <= 1e-3
        ok, k = s.solve(1e-3, 100)
        assert ok and k == 3
        assert s.stats()["sweeps"] - s.stats()["fp32_sweeps"] == 3


def test_refine_switch_keeps_the_invariant():
    n = 120
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=4, weights=(0.5, 2.0))
    with _solver(n, d, w, tile=16, precision="fp32_refine") as s:
        s.sweep(10)
        yt, yp = s.get_duals()
        s.refine_fp64()
        assert s.stats()["state_fp32"] == 0
        x, f = s.get_x()
        yt2, yp2 = s.get_duals()
    # duals are converted exactly; x and f equal the invariant evaluated by the oracle's dense rows
    np.testing.assert_array_equal(yt2, yt)
    np.testing.assert_array_equal(yp2, yp)
    from oracle import dense
    if n <= 130:
        r = dense.invariant_residual(n, d, w, 0.2, x, f, yt2, yp2)
        assert r <= 1e-12


def test_full_size_chunglu3000w_fp32_refine():
    """The weighted n = 3000 configuration in the FP32 bulk form (here on the
    sparse store, which gives the dense store's values bit for bit and keeps
    the test at about 1 GB; the oracle needs minutes per sweep at this size,
    so properties are checked): the FP64 switch rebuilds x consistently with
    the FP32 state, the refined solve reaches the tolerance, and its LP
    objective and x agree with a plain FP64 solve."""
    import paper_1901_10084_gb300 as cc
    n, d, w, _ = workload("chunglu3000w")
    with cc.Solver(n, d, w, tile=16, precision="fp32_refine", store="sparse") as s:
        s.sweep(20)
        x32, _ = s.get_x()
        s.refine_fp64()
        x64, _ = s.get_x()
        assert np.max(np.abs(x64 - x32)) <= 1e-4 * max(np.max(np.abs(x32)), 1.0)
    res = {}
    for prec in ("fp32_refine", "fp64"):
        with cc.Solver(n, d, w, tile=16, precision=prec, store="sparse", check_every=10) as s:
            conv, k = s.solve(1e-4, 3000)
            st = s.check()
            res[prec] = (conv, st, s.get_x()[0])
    for prec in res:
        assert res[prec][0] and res[prec][1]["max_violation"] <= 1e-4
    lp32, lp64 = res["fp32_refine"][1]["lp_objective"], res["fp64"][1]["lp_objective"]
    assert abs(lp32 - lp64) <= 1e-4 * abs(lp64)
    assert np.max(np.abs(res["fp32_refine"][2] - res["fp64"][2])) <= 1e-2
