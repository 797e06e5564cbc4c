"""GPU Dykstra solver for the metric-constrained LP relaxation of correlation
clustering (parallel projection method with conflict-free schedules).

The solver itself is the CUDA library ``libccdyk.so`` behind the C ABI of
``include/ccdyk.h``; ``_native`` mirrors that ABI name for name and ``Solver``
wraps it with PyTorch's stream and caching allocator.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import (CCError, CC_OK, CC_ERR_ARG, CC_ERR_OOM, CC_ERR_CUDA, CC_ERR_TIMEOUT,
                      CC_ERR_NOT_CONVERGED, CC_ERR_UNSUPPORTED, CC_ERR_BOUNDS, CC_SCHED_DIAGONAL,
                      CC_SCHED_SUMMOD, CC_SCHED_TILED, CC_PREC_FP64, CC_PREC_FP32_REFINE,
                      cc_opts_default, cc_create, cc_create_device, cc_sweep, cc_check, cc_solve,
                      cc_get_x, cc_get_duals, cc_set_state, cc_get_stats, cc_device_bytes,
                      cc_destroy, cc_last_error, cc_refine_fp64, cc_set_duals, cc_check_noalloc,
                      cc_pair_passes)
from .buildlib import build

__all__ = [
    "Solver", "Batch", "autotune_batch", "CCError", "build", "num_pairs", "num_triplets",
    "cc_opts_default", "cc_create", "cc_create_device", "cc_sweep", "cc_check", "cc_solve",
    "cc_get_x", "cc_get_duals", "cc_set_state", "cc_get_stats", "cc_device_bytes",
    "cc_destroy", "cc_last_error", "cc_refine_fp64", "cc_set_duals", "cc_check_noalloc",
    "cc_pair_passes",
]

SCHEDULES = {"diagonal": CC_SCHED_DIAGONAL, "summod": CC_SCHED_SUMMOD, "tiled": CC_SCHED_TILED}
PROBLEMS = {"cc": _native.CC_PROB_CC, "l2": _native.CC_PROB_L2}
STORES = {"dense": _native.CC_STORE_DENSE, "sparse": _native.CC_STORE_SPARSE}
PRECISIONS = {"fp64": CC_PREC_FP64, "fp32_refine": CC_PREC_FP32_REFINE}


def num_pairs(n: int) -> int:
    return n * (n - 1) // 2


def num_triplets(n: int) -> int:
    return n * (n - 1) * (n - 2) // 6


class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching
    allocator (the callbacks stay alive as long as the solver)."""

    def __init__(self, device: int):
        import torch
        self._torch = torch
        self.device = device

        def _alloc(ctx, nbytes, stream):
            # a failed request must come back as NULL (the library then reports
            # CC_ERR_OOM); an exception cannot cross the C callback
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0)))
            except Exception:
                return 0

        def _free(ctx, ptr, stream):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _native.ALLOC_FN(_alloc)
        self.free = _native.FREE_FN(_free)


class Solver:
    """One correlation-clustering LP instance (``problem="cc"``) or one l2
    metric nearness instance (``problem="l2"``: min sum w (x - d)^2 over the
    triangle inequalities) on one GPU.

    ``d`` and ``w`` are the packed pair arrays (P = n(n-1)/2 doubles, row-major
    over i<j).  ``stream`` is a ``torch.cuda.Stream`` (default: the current
    stream); with ``torch_alloc`` the device memory comes from PyTorch's
    caching allocator.
    """

    def __init__(self, n, d, w, eps=0.2, schedule="tiled", tile=16, precision="fp64",
                 exact=False, check_every=10, device=0, stream=None, torch_alloc=True,
                 barrier_timeout_s=2.0, grid=0, debug_skip_cta=-1, on_device=False, variant=-1,
                 refine_at=1e-5, trace=False, interleave=True, problem="cc", store="dense",
                 pool_entries=0, refine_sweeps=5):
        o = cc_opts_default()
        o.problem = PROBLEMS[problem] if isinstance(problem, str) else int(problem)
        o.store = STORES[store] if isinstance(store, str) else int(store)
        o.pool_entries = int(pool_entries)
        o.eps = float(eps)
        o.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        o.tile = int(tile)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.exact = 1 if exact else 0
        o.check_every = int(check_every)
        o.device = int(device)
        o.barrier_timeout_s = float(barrier_timeout_s)
        o.grid = int(grid)
        o.debug_skip_cta = int(debug_skip_cta)
        o.variant = int(variant)
        o.refine_at = float(refine_at)
        o.refine_sweeps = int(refine_sweeps)
        o.trace = 1 if trace else 0
        o.interleave = 1 if interleave else 0
        self._alloc = None
        try:
            import torch
            if stream is None:
                stream = torch.cuda.current_stream(device)
            o.stream = ctypes.c_void_p(int(stream.cuda_stream))
            self.stream = stream
            if torch_alloc:
                self._alloc = _TorchAllocator(device)
                o.alloc = self._alloc.alloc
                o.free = self._alloc.free
        except ImportError:
            self.stream = None
        self.n = int(n)
        self.eps = float(eps)
        self.opts = o
        if on_device:
            self.h = cc_create_device(self.n, int(d.data_ptr()), int(w.data_ptr()), o)
        else:
            d = np.ascontiguousarray(d, dtype=np.float64)
            w = np.ascontiguousarray(w, dtype=np.float64)
            P = num_pairs(self.n)
            if d.shape != (P,) or w.shape != (P,):
                raise ValueError(f"d and w must have {P} entries")
            self.h = cc_create(self.n, d, w, o)

    # ---- thin forwards
    def sweep(self, k: int = 1) -> None:
        cc_sweep(self.h, k)

    def pair_passes(self, passes: int) -> None:
        """Visit the pair rows alone `passes` times (see cc_pair_passes)."""
        cc_pair_passes(self.h, passes)

    def check(self) -> dict:
        return cc_check(self.h).as_dict()

    def solve(self, tol: float, max_sweeps: int) -> tuple[bool, int]:
        """Sweep until the largest metric-row violation is <= tol; returns
        (converged, sweeps run)."""
        rc, done = cc_solve(self.h, tol, max_sweeps)
        return rc == CC_OK, done

    def get_x(self):
        P = num_pairs(self.n)
        x, f = np.empty(P), np.empty(P)
        cc_get_x(self.h, x, f)
        return x, f

    def get_duals(self, first: int = 0, count: int | None = None, pairs: bool = True):
        T = num_triplets(self.n)
        if count is None:
            count = T - first
        yt = np.empty(3 * count)
        yp = np.empty(2 * num_pairs(self.n)) if pairs else None
        cc_get_duals(self.h, yt, yp, first, count)
        return yt, yp

    def set_state(self, x, f, y_tri, y_pair) -> None:
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        cc_set_state(self.h, c(x), c(f), c(y_tri), c(y_pair))

    def trace(self):
        return _native.cc_get_trace(self.h)

    def refine_fp64(self) -> None:
        cc_refine_fp64(self.h)

    def set_duals(self, y_tri, y_pair) -> None:
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        cc_set_duals(self.h, c(y_tri), c(y_pair))

    def stats(self) -> dict:
        return cc_get_stats(self.h).as_dict()

    def device_bytes(self) -> int:
        return cc_device_bytes(self.h)

    def warm_start(self, params, threshold: float = 0.0) -> int:
        """Start from the duals a trained warm-start network predicts (see
        ``warmstart``); returns the number of candidate triplets."""
        return _native.cc_warm_start_mlp(self.h, params, threshold)

    @classmethod
    def _borrow(cls, h, n, eps):
        """A view of a handle owned elsewhere (an instance of a Batch)."""
        s = cls.__new__(cls)
        s.h, s.n, s.eps, s._borrowed, s._alloc = h, int(n), float(eps), True, None
        return s

    def close(self) -> None:
        if getattr(self, "_borrowed", False):
            self.h = None
            return
        if getattr(self, "h", None) is not None:
            cc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many correlation-clustering instances of uneven size swept together:
    one launch per sweep drains the work of every active instance.

    ``instances`` is a list of (n, d, w); keyword options as for Solver (the
    tiled schedule and the fused form are required).  ``instance(i)`` gives
    a Solver view of instance i (get_x, get_duals, check, set_state ...)."""

    def __init__(self, instances, eps=0.2, tile=16, precision="fp64", check_every=10, device=0,
                 stream=None, torch_alloc=True, interleave=True, batch_order=0, grid=0, variant=0,
                 refine_sweeps=5):
        import torch
        o = cc_opts_default()
        o.eps = float(eps)
        o.tile = int(tile)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.check_every = int(check_every)
        o.device = int(device)
        o.interleave = 1 if interleave else 0
        o.batch_order = int(batch_order)
        o.grid = int(grid)
        o.variant = int(variant)
        o.refine_sweeps = int(refine_sweeps)
        if stream is None:
            stream = torch.cuda.current_stream(device)
        o.stream = ctypes.c_void_p(int(stream.cuda_stream))
        self.stream = stream
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(device)
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
        self.opts = o
        self.ns = [int(n) for n, _, _ in instances]
        self.eps = float(eps)
        self.b = _native.cc_batch_create(self.ns, [d for _, d, _ in instances], [w for _, _, w in instances], o)

    def __len__(self):
        return len(self.ns)

    def instance(self, i: int) -> Solver:
        return Solver._borrow(_native.cc_batch_handle(self.b, i), self.ns[i], self.eps)

    def sweep(self, k: int = 1) -> None:
        _native.cc_batch_sweep(self.b, k)

    def solve(self, tol: float, max_sweeps: int):
        """Returns (all converged, batch sweeps, sweeps per instance)."""
        rc, done, per = _native.cc_batch_solve(self.b, tol, max_sweeps)
        return rc == CC_OK, done, per

    def close(self) -> None:
        if getattr(self, "b", None) is not None:
            _native.cc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def autotune_batch(instances, trial_sweeps=5, **kw):
    """Pick tile, work-list order and (FP64) sweep form for a batch by timing trial sweeps;
    returns (options dict for Batch, ms per sweep)."""
    import torch
    o = cc_opts_default()
    o.eps = float(kw.get("eps", 0.2))
    o.precision = PRECISIONS[kw.get("precision", "fp64")]
    o.interleave = 1 if kw.get("interleave", True) else 0
    stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(int(stream.cuda_stream))
    best, ms = _native.cc_batch_autotune([n for n, _, _ in instances], [d for _, d, _ in instances],
                                         [w for _, _, w in instances], o, trial_sweeps)
    return {"tile": best.tile, "batch_order": best.batch_order, "variant": best.variant}, ms
