"""Device-memory failures on the GPU: an allocator that refuses the k-th
request (for every k during creation and the first sweeps) must make the
call fail with CC_ERR_OOM and leave nothing allocated; a dense store larger
than the device must be refused cleanly while the sparse store serves the
same n."""
import ctypes

import numpy as np
import pytest

from instances import chung_lu

pytestmark = pytest.mark.gpu


class FailingAllocator:
    """Pass-through to PyTorch's caching allocator that refuses request
    number `fail_at` (counting from 0; None: never) and tracks live blocks."""

    def __init__(self, fail_at=None):
        import torch
        from paper_1901_10084_gb300 import _native
        self.fail_at, self.calls, self.live = fail_at, 0, {}
        self.refuse_all = False

        def _alloc(ctx, nbytes, stream):
            k = self.calls
            self.calls += 1
            if self.refuse_all or (self.fail_at is not None and k == self.fail_at):
                return 0
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0)))
            self.live[p] = int(nbytes)
            return p

        def _free(ctx, ptr, stream):
            self.live.pop(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _native.ALLOC_FN(_alloc)
        self.free = _native.FREE_FN(_free)


def _create_and_sweep(n, d, w, alloc, **kw):
    import torch
    from paper_1901_10084_gb300 import _native as N
    o = N.cc_opts_default()
    o.alloc, o.free = alloc.alloc, alloc.free
    o.stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    for k, v in kw.items():
        setattr(o, k, v)
    h = N.cc_create(n, d, w, o)
    try:
        N.cc_sweep(h, 3)
        N.cc_check(h)
        if o.precision == N.CC_PREC_FP32_REFINE:
            N.cc_refine_fp64(h)      # the switch allocates the FP64 state
            N.cc_sweep(h, 1)
        x = np.empty(len(d))
        N.cc_get_x(h, x, None)
        yt = np.empty(3 * (n * (n - 1) * (n - 2) // 6))
        N.cc_get_duals(h, yt, None)
    finally:
        N.cc_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("store", [0, 1])
def test_every_allocation_failure_is_reported_and_cleaned_up(store, precision):
    """Creation, sweeps (with a one-entry starting pool the sparse store grows
    its pools during the sweeps), the check, the read-backs and, in the FP32
    bulk form, the switch to FP64."""
    from paper_1901_10084_gb300 import _native as N
    n = 70
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=4)
    kw = dict(store=store, precision=precision, pool_entries=1 if store else 0)
    ref = FailingAllocator()
    _create_and_sweep(n, d, w, ref, **kw)
    assert ref.calls > 5 and not ref.live
    for k in range(ref.calls):
        a = FailingAllocator(fail_at=k)
        with pytest.raises(N.CCError) as e:
            _create_and_sweep(n, d, w, a, **kw)
        assert e.value.code == N.CC_ERR_OOM, k
        assert not a.live, (k, a.live)


def test_dense_store_beyond_the_device_is_refused_and_the_sparse_store_serves():
    import paper_1901_10084_gb300 as cc
    n = 6000   # dense FP64 triangle store: 3 C(n,3) x 8 B = 863 GB
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=5)
    with pytest.raises(cc.CCError) as e:
        cc.Solver(n, d, w, tile=16)
    assert e.value.code == cc.CC_ERR_OOM
    with cc.Solver(n, d, w, tile=16, store="sparse") as s:
        s.sweep(2)
        assert s.check()["max_violation"] >= 0.0
        assert s.device_bytes() < 16e9



def test_sweeps_after_a_failed_pool_growth():
    """The next pool cannot grow: the sweep is undone and reports
    CC_ERR_OOM; while memory stays short every further sweep does the same
    (nothing is written to a pool that is gone); once memory is back the
    sweeps go on and give the values of an undisturbed run."""
    import torch
    from paper_1901_10084_gb300 import _native as N
    n = 70
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=4)

    def handle(alloc):
        o = N.cc_opts_default()
        o.alloc, o.free = alloc.alloc, alloc.free
        o.stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
        o.store, o.pool_entries = 1, 1
        return N.cc_create(n, d, w, o)

    ref_alloc = FailingAllocator()
    ref = handle(ref_alloc)
    N.cc_sweep(ref, 4)
    x_ref = np.empty(len(d))
    N.cc_get_x(ref, x_ref, None)
    N.cc_destroy(ref)

    a = FailingAllocator()
    h = handle(a)
    try:
        N.cc_sweep(h, 1)                    # the first sweep writes no entries
        a.refuse_all = True
        for _ in range(2):
            with pytest.raises(N.CCError) as e:
                N.cc_sweep(h, 1)
            assert e.value.code == N.CC_ERR_OOM
        a.refuse_all = False
        N.cc_sweep(h, 3)
        x = np.empty(len(d))
        N.cc_get_x(h, x, None)
        assert np.array_equal(x, x_ref)
    finally:
        N.cc_destroy(h)
    assert not a.live and not ref_alloc.live
