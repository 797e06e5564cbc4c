"""ctypes binding of the C ABI in include/ccdyk.h (argument marshalling only).

Every function here forwards to libccdyk.so under the same name; all solver
work runs in that library's CUDA kernels.  Loading fails loudly when the
library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import buildlib as _build

CC_OK = 0
CC_ERR_ARG = 1
CC_ERR_OOM = 2
CC_ERR_CUDA = 3
CC_ERR_TIMEOUT = 4
CC_ERR_NOT_CONVERGED = 5
CC_ERR_UNSUPPORTED = 6
CC_ERR_BOUNDS = 7

CC_SCHED_DIAGONAL = 0
CC_SCHED_SUMMOD = 1
CC_SCHED_TILED = 2

CC_PREC_FP64 = 0
CC_PREC_FP32_REFINE = 1

CC_PROB_CC = 0
CC_PROB_L2 = 1

CC_STORE_DENSE = 0
CC_STORE_SPARSE = 1

CC_NOALLOC_MAX_N = 4096

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class cc_opts(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.c_double),
        ("schedule", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("exact", ctypes.c_int32),
        ("check_every", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("barrier_timeout_s", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("grid", ctypes.c_int32),
        ("debug_skip_cta", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("refine_at", ctypes.c_double),
        ("trace", ctypes.c_int32),
        ("interleave", ctypes.c_int32),
        ("batch_order", ctypes.c_int32),
        ("problem", ctypes.c_int32),
        ("store", ctypes.c_int32),
        ("pool_entries", ctypes.c_int64),
        ("refine_sweeps", ctypes.c_int32),
    ]


class cc_stats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int64),
        ("max_violation", ctypes.c_double),
        ("pair_violation", ctypes.c_double),
        ("lp_objective", ctypes.c_double),
        ("wf", ctypes.c_double),
        ("qp_primal", ctypes.c_double),
        ("dual_objective", ctypes.c_double),
        ("gap", ctypes.c_double),
        ("last_sweep_ms", ctypes.c_double),
        ("fp32_sweeps", ctypes.c_int64),
        ("state_fp32", ctypes.c_int32),
        ("dual_nnz", ctypes.c_int64),
        ("pool_retries", ctypes.c_int64),
        ("variant", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ("cc_opts_default", "cc_create", "cc_create_device", "cc_sweep", "cc_check",
           "cc_solve", "cc_get_x", "cc_get_duals", "cc_set_state", "cc_get_stats",
           "cc_device_bytes", "cc_destroy", "cc_last_error", "cc_check_noalloc",
           "cc_refine_fp64", "cc_set_duals", "cc_get_trace", "cc_batch_create", "cc_batch_size",
           "cc_batch_handle", "cc_batch_sweep", "cc_batch_solve", "cc_batch_autotune", "cc_batch_destroy",
           "cc_batch_last_error", "cc_warm_start_mlp", "cc_ws_samples", "cc_mlp_forward", "cc_mlp_grad",
           "cc_mlp_train", "cc_pair_passes")

CC_WS_NPARAM = 5059
CC_WS_FEAT = 12
CC_WS_PAIR_PASSES = 16

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    """libccdyk.so, or libccdyk_checked.so when CCDYK_CHECKED=1."""
    return _build.LIB_CHECKED if os.environ.get("CCDYK_CHECKED") == "1" else _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libccdyk.so; raise if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"{os.path.basename(path)} not built at {path}; run __graft_entry__.build() "
                "(the CUDA library is the only implementation)")
        lib = ctypes.CDLL(path)
        H = ctypes.c_void_p
        HP = ctypes.POINTER(ctypes.c_void_p)
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.cc_opts_default.argtypes = [ctypes.POINTER(cc_opts)]
        lib.cc_opts_default.restype = None
        lib.cc_create.argtypes = [HP, i64, dp, dp, ctypes.POINTER(cc_opts)]
        lib.cc_create.restype = ctypes.c_int
        lib.cc_create_device.argtypes = [HP, i64, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(cc_opts)]
        lib.cc_create_device.restype = ctypes.c_int
        lib.cc_sweep.argtypes = [H, i64]
        lib.cc_sweep.restype = ctypes.c_int
        lib.cc_pair_passes.argtypes = [H, ctypes.c_int32]
        lib.cc_pair_passes.restype = ctypes.c_int
        lib.cc_check.argtypes = [H, ctypes.POINTER(cc_stats)]
        lib.cc_check.restype = ctypes.c_int
        lib.cc_solve.argtypes = [H, ctypes.c_double, i64, ctypes.POINTER(ctypes.c_int64)]
        lib.cc_solve.restype = ctypes.c_int
        lib.cc_get_x.argtypes = [H, dp, dp]
        lib.cc_get_x.restype = ctypes.c_int
        lib.cc_get_duals.argtypes = [H, dp, dp, i64, i64]
        lib.cc_get_duals.restype = ctypes.c_int
        lib.cc_set_state.argtypes = [H, dp, dp, dp, dp]
        lib.cc_set_state.restype = ctypes.c_int
        lib.cc_get_stats.argtypes = [H, ctypes.POINTER(cc_stats)]
        lib.cc_get_stats.restype = ctypes.c_int
        lib.cc_device_bytes.argtypes = [H]
        lib.cc_device_bytes.restype = i64
        lib.cc_destroy.argtypes = [H]
        lib.cc_destroy.restype = None
        lib.cc_last_error.argtypes = [H]
        lib.cc_last_error.restype = ctypes.c_char_p
        PP = ctypes.POINTER(ctypes.c_void_p)
        I64P = ctypes.POINTER(ctypes.c_int64)
        lib.cc_batch_create.argtypes = [HP, ctypes.c_int32, I64P, PP, PP, ctypes.POINTER(cc_opts)]
        lib.cc_batch_create.restype = ctypes.c_int
        lib.cc_batch_size.argtypes = [H]
        lib.cc_batch_size.restype = ctypes.c_int32
        lib.cc_batch_handle.argtypes = [H, ctypes.c_int32]
        lib.cc_batch_handle.restype = ctypes.c_void_p
        lib.cc_batch_sweep.argtypes = [H, i64]
        lib.cc_batch_sweep.restype = ctypes.c_int
        lib.cc_batch_solve.argtypes = [H, ctypes.c_double, i64, I64P, I64P]
        lib.cc_batch_solve.restype = ctypes.c_int
        lib.cc_batch_autotune.argtypes = [ctypes.c_int32, I64P, PP, PP, ctypes.POINTER(cc_opts), ctypes.c_int32,
                                          ctypes.POINTER(cc_opts), ctypes.POINTER(ctypes.c_double)]
        lib.cc_batch_autotune.restype = ctypes.c_int
        lib.cc_batch_destroy.argtypes = [H]
        lib.cc_batch_destroy.restype = None
        lib.cc_batch_last_error.argtypes = [H]
        lib.cc_batch_last_error.restype = ctypes.c_char_p
        lib.cc_get_trace.argtypes = [H, ctypes.POINTER(ctypes.c_uint64), i64]
        lib.cc_get_trace.restype = i64
        lib.cc_refine_fp64.argtypes = [H]
        lib.cc_refine_fp64.restype = ctypes.c_int
        lib.cc_set_duals.argtypes = [H, dp, dp]
        lib.cc_set_duals.restype = ctypes.c_int
        vp = ctypes.c_void_p
        lib.cc_check_noalloc.argtypes = [i64, ctypes.c_double, vp, vp, vp, vp, vp, vp, vp]
        lib.cc_check_noalloc.restype = ctypes.c_int
        fp = ctypes.POINTER(ctypes.c_float)
        lib.cc_warm_start_mlp.argtypes = [H, fp, ctypes.c_double, I64P]
        lib.cc_warm_start_mlp.restype = ctypes.c_int
        lib.cc_ws_samples.argtypes = [H, vp, vp, i64, I64P]
        lib.cc_ws_samples.restype = ctypes.c_int
        lib.cc_mlp_forward.argtypes = [fp, vp, vp, i64, vp]
        lib.cc_mlp_forward.restype = ctypes.c_int
        lib.cc_mlp_grad.argtypes = [fp, vp, vp, i64, ctypes.c_float, fp, fp, vp]
        lib.cc_mlp_grad.restype = ctypes.c_int
        lib.cc_mlp_train.argtypes = [fp, vp, vp, i64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                     ctypes.c_uint64, ctypes.c_float, fp, vp]
        lib.cc_mlp_train.restype = ctypes.c_int
        _lib = lib
        return lib


class CCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, h) -> None:
    if rc != CC_OK:
        msg = load().cc_last_error(h)
        raise CCError(rc, msg.decode() if msg else "")


# ---- same names as the C ABI ---------------------------------------------

def cc_opts_default() -> cc_opts:
    o = cc_opts()
    load().cc_opts_default(ctypes.byref(o))
    return o


def cc_create(n: int, d, w, opts: cc_opts | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    rc = load().cc_create(ctypes.byref(h), n, _dp(d), _dp(w), ctypes.byref(opts) if opts else None)
    _check(rc, None)
    return h


def cc_create_device(n: int, d_ptr: int, w_ptr: int, opts: cc_opts | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    rc = load().cc_create_device(ctypes.byref(h), n, ctypes.c_void_p(d_ptr), ctypes.c_void_p(w_ptr),
                                 ctypes.byref(opts) if opts else None)
    _check(rc, None)
    return h


def cc_sweep(h, k: int) -> None:
    _check(load().cc_sweep(h, k), h)


def cc_pair_passes(h, passes: int) -> None:
    _check(load().cc_pair_passes(h, passes), h)


def cc_check(h) -> cc_stats:
    st = cc_stats()
    _check(load().cc_check(h, ctypes.byref(st)), h)
    return st


def cc_solve(h, tol: float, max_sweeps: int) -> tuple[int, int]:
    """Returns (status, sweeps_done); status is CC_OK or CC_ERR_NOT_CONVERGED."""
    done = ctypes.c_int64(0)
    rc = load().cc_solve(h, tol, max_sweeps, ctypes.byref(done))
    if rc not in (CC_OK, CC_ERR_NOT_CONVERGED):
        _check(rc, h)
    return rc, done.value


def cc_get_x(h, x, f=None) -> None:
    _check(load().cc_get_x(h, _dp(x), _dp(f)), h)


def cc_get_duals(h, y_tri, y_pair, tri_first: int = 0, tri_count: int = 0) -> None:
    _check(load().cc_get_duals(h, _dp(y_tri), _dp(y_pair), tri_first, tri_count), h)


def cc_set_state(h, x, f, y_tri, y_pair) -> None:
    _check(load().cc_set_state(h, _dp(x), _dp(f), _dp(y_tri), _dp(y_pair)), h)


def cc_get_trace(h):
    """Per-item timestamps of the last fused tiled sweep as an (items, 6)
    uint64 array (empty when tracing is off)."""
    import numpy as np
    items = int(load().cc_get_trace(h, None, 0))
    out = np.zeros((max(items, 0), 6), dtype=np.uint64)
    if items > 0:
        got = load().cc_get_trace(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), items)
        if got < 0:
            raise CCError(CC_ERR_CUDA, "cc_get_trace failed")
    return out


def cc_refine_fp64(h) -> None:
    _check(load().cc_refine_fp64(h), h)


def cc_set_duals(h, y_tri, y_pair) -> None:
    _check(load().cc_set_duals(h, _dp(y_tri), _dp(y_pair)), h)


def cc_get_stats(h) -> cc_stats:
    st = cc_stats()
    _check(load().cc_get_stats(h, ctypes.byref(st)), h)
    return st


def cc_device_bytes(h) -> int:
    return int(load().cc_device_bytes(h))


def cc_destroy(h) -> None:
    load().cc_destroy(h)


def cc_last_error(h=None) -> str:
    m = load().cc_last_error(h)
    return m.decode() if m else ""


def cc_check_noalloc(n: int, eps: float, x_ptr: int, f_ptr: int, d_ptr: int, w_ptr: int,
                     y_pair_ptr: int, out_ptr: int, stream: int = 0) -> int:
    """Convergence check from caller-owned device arrays (packed layouts) into
    a caller-owned device array of 8 doubles; allocates nothing.  Returns the
    status code (CC_OK or an error; message in cc_last_error())."""
    v = ctypes.c_void_p
    return int(load().cc_check_noalloc(n, eps, v(x_ptr), v(f_ptr), v(d_ptr), v(w_ptr),
                                       v(y_pair_ptr), v(out_ptr), v(stream)))


# ---- batches ---------------------------------------------------------------

def _batch_arrays(ns, ds, ws):
    import numpy as np
    count = len(ns)
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in list(ds) + list(ws)]
    n_arr = (ctypes.c_int64 * count)(*[int(v) for v in ns])
    d_arr = (ctypes.c_void_p * count)(*[a.ctypes.data for a in keep[:count]])
    w_arr = (ctypes.c_void_p * count)(*[a.ctypes.data for a in keep[count:]])
    return count, n_arr, d_arr, w_arr, keep


def _bcheck(rc: int, b) -> None:
    if rc != CC_OK:
        msg = load().cc_batch_last_error(b)
        raise CCError(rc, msg.decode() if msg else "")


def cc_batch_create(ns, ds, ws, opts: cc_opts | None = None):
    count, n_arr, d_arr, w_arr, keep = _batch_arrays(ns, ds, ws)
    b = ctypes.c_void_p()
    rc = load().cc_batch_create(ctypes.byref(b), count, n_arr, d_arr, w_arr,
                                ctypes.byref(opts) if opts else None)
    _bcheck(rc, None)
    return b


def cc_batch_size(b) -> int:
    return int(load().cc_batch_size(b))


def cc_batch_handle(b, i: int):
    return ctypes.c_void_p(load().cc_batch_handle(b, i))


def cc_batch_sweep(b, k: int) -> None:
    _bcheck(load().cc_batch_sweep(b, k), b)


def cc_batch_solve(b, tol: float, max_sweeps: int):
    """Returns (status, batch sweeps, sweeps per instance)."""
    count = cc_batch_size(b)
    per = (ctypes.c_int64 * count)()
    done = ctypes.c_int64(0)
    rc = load().cc_batch_solve(b, tol, max_sweeps, ctypes.byref(done), per)
    if rc not in (CC_OK, CC_ERR_NOT_CONVERGED):
        _bcheck(rc, b)
    return rc, done.value, list(per)


def cc_batch_autotune(ns, ds, ws, base: cc_opts | None, trial_sweeps: int):
    count, n_arr, d_arr, w_arr, keep = _batch_arrays(ns, ds, ws)
    best = cc_opts()
    ms = ctypes.c_double(0.0)
    rc = load().cc_batch_autotune(count, n_arr, d_arr, w_arr, ctypes.byref(base) if base else None,
                                  trial_sweeps, ctypes.byref(best), ctypes.byref(ms))
    _bcheck(rc, None)
    return best, ms.value


def cc_batch_destroy(b) -> None:
    load().cc_batch_destroy(b)


def cc_batch_last_error(b=None) -> str:
    m = load().cc_batch_last_error(b)
    return m.decode() if m else ""


# ---- learned dual warm start -------------------------------------------------

def _fp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _params(p):
    import numpy as np
    a = np.ascontiguousarray(p, dtype=np.float32)
    if a.shape != (CC_WS_NPARAM,):
        raise ValueError(f"params must hold {CC_WS_NPARAM} floats")
    return a


def cc_warm_start_mlp(h, params, threshold: float) -> int:
    """Replace the duals by the network's prediction; returns the number of
    candidate triplets."""
    p = _params(params)
    cand = ctypes.c_int64(0)
    _check(load().cc_warm_start_mlp(h, _fp(p), threshold, ctypes.byref(cand)), h)
    return cand.value


def cc_ws_samples(h, feat_ptr: int = 0, target_ptr: int = 0, cap: int = 0) -> int:
    """Candidate count; with device pointers also writes features and targets."""
    cnt = ctypes.c_int64(0)
    v = ctypes.c_void_p
    _check(load().cc_ws_samples(h, v(feat_ptr) if feat_ptr else None, v(target_ptr) if target_ptr else None,
                                cap, ctypes.byref(cnt)), h)
    return cnt.value


def cc_mlp_forward(params, feat_ptr: int, out_ptr: int, count: int, stream: int = 0) -> None:
    p = _params(params)
    v = ctypes.c_void_p
    _check(load().cc_mlp_forward(_fp(p), v(feat_ptr), v(out_ptr), count, v(stream)), None)


def cc_mlp_grad(params, feat_ptr: int, target_ptr: int, count: int, pos_weight: float = 1.0, stream: int = 0):
    """Returns (gradient as float32 array, loss)."""
    import numpy as np
    p = _params(params)
    g = np.zeros(CC_WS_NPARAM, dtype=np.float32)
    loss = ctypes.c_float(0.0)
    v = ctypes.c_void_p
    _check(load().cc_mlp_grad(_fp(p), v(feat_ptr), v(target_ptr), count, pos_weight, _fp(g), ctypes.byref(loss),
                              v(stream)),
           None)
    return g, float(loss.value)


def cc_mlp_train(params, feat_ptr: int, target_ptr: int, count: int, batch: int, steps: int, lr: float,
                 seed: int, pos_weight: float = 1.0, stream: int = 0):
    """Returns (trained params, per-step minibatch losses); params is not modified."""
    import numpy as np
    p = _params(params).copy()
    losses = np.zeros(max(steps, 0), dtype=np.float32)
    v = ctypes.c_void_p
    _check(load().cc_mlp_train(_fp(p), v(feat_ptr), v(target_ptr), count, batch, steps, lr, seed, pos_weight,
                               _fp(losses) if steps > 0 else None, v(stream)), None)
    return p, losses
