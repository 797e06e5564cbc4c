"""cc_check_noalloc: the convergence check for callers that cannot allocate
device memory when they need it (device memory reserved in full by another
allocator, or a loop that cannot afford cudaMalloc's device synchronization).
Its scratch is a fixed array inside the library, so its result must match
cc_check on a handle (which uses scratch the handle allocated) on consecutive
calls, with the array keeping whatever the previous call left in it.

Its results are also compared with the oracle's definitions of the same
quantities (the largest metric-row violation over every triplet, the
objective sums) at n = 1000 on an oracle Dykstra state and at the largest n
it accepts on seeded arrays.

This file is collected last so that a run stopping at the first failure has
run every other test first."""
import numpy as np
import pytest

from instances import planted_partition, chung_lu


@pytest.mark.gpu
def test_check_noalloc_matches_cc_check_on_two_calls_in_a_row():
    import torch

    import paper_1901_10084_gb300 as cc
    from paper_1901_10084_gb300 import _native as N

    def run(n, d, w, sweeps, exact):
        with cc.Solver(n, d, w, eps=0.25, tile=16, exact=exact) as s:
            s.sweep(sweeps)
            st = s.check()
            x, f = s.get_x()
            _, yp = s.get_duals(0, 0)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        tx, tf, td, tw, typ = dev(x), dev(f), dev(d), dev(w), dev(yp)
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        rc = N.cc_check_noalloc(n, 0.25, tx.data_ptr(), tf.data_ptr(), td.data_ptr(), tw.data_ptr(),
                                typ.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == N.CC_OK, N.cc_last_error()
        got = out.cpu().numpy()
        assert got[0] == st["max_violation"]                     # a maximum is order-free: exact
        assert got[1] == pytest.approx(st["pair_violation"], abs=1e-15)
        for k, name in ((2, "lp_objective"), (3, "wf"), (4, "qp_primal"), (5, "dual_objective"),
                        (6, "gap")):
            assert got[k] == pytest.approx(st[name], rel=1e-12, abs=1e-10)

    # first call: larger instance; second call: smaller one, so rows the
    # first call wrote beyond the second's n stay in the array unread
    d1, w1, _ = chung_lu(300, 2.5, 8.0, seed=5, weights=(0.5, 2.0))
    run(300, d1, w1, 6, exact=False)
    d2, w2, _ = planted_partition(130, 4, 0.8, 0.1, seed=6)
    run(130, d2, w2, 3, exact=True)


def test_check_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1901_10084_gb300 import _native as N
    N.load(build_if_missing=True)
    big = 4097
    rc = N.cc_check_noalloc(big, 0.2, 16, 16, 16, 16, 16, 16, 0)  # rejected before any device access
    assert rc == N.CC_ERR_ARG
    assert "CC_NOALLOC_MAX_N" in N.cc_last_error()
    assert N.cc_check_noalloc(2, 0.2, 16, 16, 16, 16, 16, 16, 0) == N.CC_ERR_ARG
    assert N.cc_check_noalloc(100, 0.2, 0, 16, 16, 16, 16, 16, 0) == N.CC_ERR_ARG


def _noalloc(n, eps, x, f, d, w, yp):
    import torch

    from paper_1901_10084_gb300 import _native as N
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    tx, tf, td, tw, typ = dev(x), dev(f), dev(d), dev(w), dev(yp)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    rc = N.cc_check_noalloc(n, eps, tx.data_ptr(), tf.data_ptr(), td.data_ptr(), tw.data_ptr(),
                            typ.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == N.CC_OK, N.cc_last_error()
    return out.cpu().numpy()


def _against_oracle(got, n, eps, x, f, d, w, yp, threads):
    """The maxima exactly (same row formulas; a maximum is order-free).  The
    sums are taken in different orders on the two sides; each is within
    (P - 1) u S of the exact sum (u = 2^-53, S the sum of the magnitudes of
    its P terms), so they may differ by 2 P u S."""
    import oracle
    mv = oracle.max_violation(n, x, threads=threads)
    oo = oracle.objectives(n, eps, d, w, x, f, yp)
    assert got[0] == mv
    assert got[1] == pytest.approx(oo["pair_violation"], abs=1e-15)
    P = x.size
    s_lp = np.sum(np.abs(w * np.abs(x - d)))
    s_wf = np.sum(np.abs(w * f))
    s_quad = np.sum(w * (x * x + f * f))
    s_by = np.sum(np.abs(d * (yp[0::2] - yp[1::2])))
    mag = {"lp": s_lp, "wf": s_wf, "qp_primal": s_wf + 0.5 * eps * s_quad, "dual": s_by + 0.5 * eps * s_quad,
           "gap": s_wf + s_by + eps * s_quad}
    for k, name in ((2, "lp"), (3, "wf"), (4, "qp_primal"), (5, "dual"), (6, "gap")):
        assert abs(got[k] - oo[name]) <= 2 * P * 2.0 ** -53 * mag[name] + 1e-300, name


@pytest.mark.gpu
def test_check_noalloc_matches_the_oracle_at_n1000_and_at_its_largest_n():
    import os

    import oracle
    threads = len(os.sched_getaffinity(0))
    # n = 1000: the oracle's own Dykstra state after three sweeps
    n, eps = 1000, 0.2
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=1)
    st = oracle.State(n, d, w, eps)
    for _ in range(3):
        st.sweep_threads(2, 16, threads)
    got = _noalloc(n, eps, st.x, st.f, d, w, st.ypair)
    _against_oracle(got, n, eps, st.x, st.f, d, w, st.ypair, threads)
    del st
    # n = CC_NOALLOC_MAX_N (4096): seeded arrays near a feasible point (the
    # oracle's dual storage at this n would need 275 GB, and the check's
    # quantities are defined for any arrays); two calls in a row
    from paper_1901_10084_gb300 import _native as N
    n = N.CC_NOALLOC_MAX_N
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=2, weights=(0.5, 2.0))
    rng = np.random.default_rng(4096)
    P = d.size
    x = 0.9 * d + rng.uniform(0.0, 0.1, P)
    f = np.abs(x - d) + rng.uniform(-1e-3, 1e-3, P)
    yp = rng.exponential(0.1, 2 * P)
    for _ in range(2):
        got = _noalloc(n, 0.3, x, f, d, w, yp)
        _against_oracle(got, n, 0.3, x, f, d, w, yp, threads)
