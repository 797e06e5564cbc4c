"""cc_check_noalloc: the convergence check for callers that cannot allocate
device memory when they need it (device memory reserved in full by another
allocator, or a loop that cannot afford cudaMalloc's device synchronization).
Its scratch is a fixed array inside the library, so its result must match
cc_check on a handle (which uses scratch the handle allocated) on consecutive
calls, with the array keeping whatever the previous call left in it.

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
