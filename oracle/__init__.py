"""Oracle for Dykstra's method on the regularized correlation-clustering LP.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  The
product path (``paper_1901_10084_gb300``) never imports it and shares no code
with it.

``dykstra.c`` is a plain serial FP64 transcription of Algorithm 1 specialised
to the metric rows of Eq. (mn1) (Sec. II-B) and walked in the schedules of
Sec. III-B/C, with a threaded form of the same sweep that deals the disjoint
units of each phase to host threads (the parallelism of Sec. III-A/C; the
result equals the serial sweep bit for bit); ``dense.py`` holds brute-force checks built from a dense
constraint matrix (an LP solve with HiGHS, A^T y, a KKT certificate).

Parity status of each function:
  * ``sweep`` / ``visit_triplet`` / ``visit_pair``: pinned (halfspace
    projection property, the worked triangle case of Sec. II-B, the invariant
    v = v0 - W^{-1} A^T y / eps, monotone dual objective, KKT at convergence,
    dense LP at small n, the closed-form clustered instance).
  * ``sweep_threads``: pinned to the serial sweep, bit for bit, for every
    schedule, thread count and partial sweep in ``tests/test_oracle_threads.py``.
  * ``order`` / ``num_phases``: pinned (brute-force coverage and
    conflict-freeness, the phase counts and set sizes the paper states).
  * ``max_violation`` / ``objectives``: pinned by direct definition checks
    against the dense constraint matrix; the threaded ``max_violation`` is
    pinned to the serial one (equal values) in ``tests/test_oracle_threads.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dykstra.c")
_LIB = os.path.join(_HERE, "_build", "libccoracle.so")
_lock = threading.Lock()
_lib = None

SCHEDULES = (0, 1, 2)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-pthread",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.ora_trank.argtypes = [i64, i64, i64, i64]
        lib.ora_trank.restype = i64
        lib.ora_pidx.argtypes = [i64, i64, i64]
        lib.ora_pidx.restype = i64
        lib.ora_init.argtypes = [i64, dbl, dp, dp, dp, dp, dp, dp]
        lib.ora_init.restype = None
        lib.ora_visit_triplet.argtypes = [i64, dbl, dp, dp, dp, i64, i64, i64, i32]
        lib.ora_visit_triplet.restype = None
        lib.ora_visit_pair.argtypes = [i64, dbl, dp, dp, dp, dp, dp, i64, i32]
        lib.ora_visit_pair.restype = None
        lib.ora_order.argtypes = [i64, i32, i64, ip, i64]
        lib.ora_order.restype = i64
        lib.ora_num_phases.argtypes = [i64, i32, i64]
        lib.ora_num_phases.restype = i64
        lib.ora_sweep.argtypes = [i64, i32, i64, dbl, dp, dp, dp, dp, dp, dp, i64]
        lib.ora_sweep.restype = i64
        lib.ora_max_violation.argtypes = [i64, dp]
        lib.ora_max_violation.restype = dbl
        lib.ora_objectives.argtypes = [i64, dbl, dp, dp, dp, dp, dp, dp]
        lib.ora_objectives.restype = None
        lib.ora_init_l2.argtypes = [i64, dp, dp, dp, dp, dp]
        lib.ora_init_l2.restype = None
        lib.ora_sweep_l2.argtypes = [i64, i32, i64, dp, dp, dp, i64]
        lib.ora_sweep_l2.restype = i64
        lib.ora_objectives_l2.argtypes = [i64, dp, dp, dp, dp]
        lib.ora_objectives_l2.restype = None
        lib.ora_sweep_threads.argtypes = [i64, i32, i64, dbl, dp, dp, dp, dp, dp, dp, i32, i64]
        lib.ora_sweep_threads.restype = i64
        lib.ora_sweep_l2_threads.argtypes = [i64, i32, i64, dp, dp, dp, i32, i64]
        lib.ora_sweep_l2_threads.restype = i64
        lib.ora_max_violation_threads.argtypes = [i64, dp, i32]
        lib.ora_max_violation_threads.restype = dbl
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_pairs(n: int) -> int:
    return n * (n - 1) // 2


def num_triplets(n: int) -> int:
    return n * (n - 1) * (n - 2) // 6


def pidx(n: int, i: int, j: int) -> int:
    return int(_load().ora_pidx(n, i, j))


def trank(n: int, i: int, j: int, k: int) -> int:
    return int(_load().ora_trank(n, i, j, k))


class State:
    """Oracle state: x, f (packed pairs), y_tri (canonical), y_pair.

    problem "cc": the regularized CC LP (Eq. mn1 as Eq. qp, parameter eps);
    problem "l2": l2 metric nearness, min sum w (x - d)^2 over the metric rows
    (Eq. metricnear, p = 2; Eq. qp with eps = 1, c = -W d; f and y_pair stay 0)."""

    def __init__(self, n: int, d: np.ndarray, w: np.ndarray, eps: float = 1.0, problem: str = "cc"):
        if problem not in ("cc", "l2"):
            raise ValueError(problem)
        self.problem = problem
        self.n = int(n)
        self.eps = float(eps) if problem == "cc" else 1.0
        P, T = num_pairs(n), num_triplets(n)
        self.d = np.ascontiguousarray(d, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        assert self.d.shape == (P,) and self.w.shape == (P,)
        self.winv = np.empty(P)
        self.x = np.empty(P)
        self.f = np.empty(P)
        self.ytri = np.empty(3 * T)
        self.ypair = np.empty(2 * P)
        if problem == "cc":
            _load().ora_init(n, self.eps, _dp(self.w), _dp(self.winv), _dp(self.x),
                             _dp(self.f), _dp(self.ytri), _dp(self.ypair))
        else:
            _load().ora_init_l2(n, _dp(self.d), _dp(self.w), _dp(self.winv), _dp(self.x),
                                _dp(self.ytri))
            self.f[:] = 0.0
            self.ypair[:] = 0.0

    def copy(self) -> "State":
        s = State.__new__(State)
        s.n, s.eps, s.problem = self.n, self.eps, self.problem
        for k in ("d", "w", "winv", "x", "f", "ytri", "ypair"):
            setattr(s, k, getattr(self, k).copy())
        return s

    def sweep(self, schedule: int = 1, tile: int = 16, max_rows: int = -1) -> int:
        """One pass over all rows in the schedule's order (or its first
        ``max_rows`` rows).  Returns the number of rows visited."""
        if self.problem == "l2":
            return int(_load().ora_sweep_l2(self.n, schedule, tile, _dp(self.winv), _dp(self.x),
                                            _dp(self.ytri), max_rows))
        return int(_load().ora_sweep(self.n, schedule, tile, self.eps, _dp(self.d),
                                     _dp(self.winv), _dp(self.x), _dp(self.f),
                                     _dp(self.ytri), _dp(self.ypair), max_rows))

    def sweep_threads(self, schedule: int = 1, tile: int = 16, threads: int = 0,
                      max_phases: int = 0) -> int:
        """The sweep with the units of each phase dealt to ``threads`` host
        threads (0: all cores); with ``max_phases`` > 0 only the metric rows
        of the first ``max_phases`` phases.  Returns the rows visited."""
        t = threads if threads > 0 else (os.cpu_count() or 1)
        if self.problem == "l2":
            r = _load().ora_sweep_l2_threads(self.n, schedule, tile, _dp(self.winv), _dp(self.x),
                                             _dp(self.ytri), t, max_phases)
        else:
            r = _load().ora_sweep_threads(self.n, schedule, tile, self.eps, _dp(self.d),
                                          _dp(self.winv), _dp(self.x), _dp(self.f),
                                          _dp(self.ytri), _dp(self.ypair), t, max_phases)
        if r < 0:
            raise RuntimeError("could not start the oracle's threads")
        return int(r)

    def visit_triplet(self, i: int, j: int, k: int, rows: int = 3) -> None:
        _load().ora_visit_triplet(self.n, self.eps, _dp(self.winv), _dp(self.x),
                                  _dp(self.ytri), i, j, k, rows)

    def visit_pair(self, p: int, rows: int = 2) -> None:
        _load().ora_visit_pair(self.n, self.eps, _dp(self.d), _dp(self.winv),
                               _dp(self.x), _dp(self.f), _dp(self.ypair), p, rows)

    def max_violation(self) -> float:
        return float(_load().ora_max_violation(self.n, _dp(self.x)))

    def objectives(self) -> dict:
        """cc: lp = sum w |x - d|; l2: lp = sum w (x - d)^2 (the problem's
        objective), qp_primal / dual / gap of the respective Eq. qp."""
        out = np.zeros(5)
        if self.problem == "l2":
            _load().ora_objectives_l2(self.n, _dp(self.d), _dp(self.w), _dp(self.x), _dp(out))
        else:
            _load().ora_objectives(self.n, self.eps, _dp(self.d), _dp(self.w), _dp(self.x),
                                   _dp(self.f), _dp(self.ypair), _dp(out))
        return {"lp": out[0], "qp_primal": out[1], "dual": out[2],
                "pair_violation": out[3], "wf": out[4], "gap": out[1] - out[2]}

    def solve(self, tol: float, max_sweeps: int, schedule: int = 1, tile: int = 16,
              check_every: int = 1) -> int:
        """Sweep until the largest metric-row violation is <= tol."""
        for s in range(1, max_sweeps + 1):
            self.sweep(schedule, tile)
            if s % check_every == 0 and self.max_violation() <= tol:
                return s
        return -1


def max_violation(n: int, x: np.ndarray, threads: int = 1) -> float:
    """Largest metric-row violation max(0, x_h - x_a - x_b) over every
    triplet and hypotenuse of the packed distances x (no State, so no dual
    storage); with ``threads`` > 1 the first indices are dealt to host
    threads (a maximum is order-free: the same value)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (num_pairs(n),)
    if threads <= 1:
        return float(_load().ora_max_violation(n, _dp(x)))
    m = float(_load().ora_max_violation_threads(n, _dp(x), threads))
    if m < 0:
        raise RuntimeError("could not start the oracle's threads")
    return m


def objectives(n: int, eps: float, d, w, x, f, ypair) -> dict:
    """The CC objectives of State.objectives on given arrays (packed pairs;
    ypair 2 per pair)."""
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    d, w, x, f, ypair = c(d), c(w), c(x), c(f), c(ypair)
    out = np.zeros(5)
    _load().ora_objectives(n, float(eps), _dp(d), _dp(w), _dp(x), _dp(f), _dp(ypair), _dp(out))
    return {"lp": out[0], "qp_primal": out[1], "dual": out[2],
            "pair_violation": out[3], "wf": out[4], "gap": out[1] - out[2]}


def order(n: int, schedule: int, tile: int = 16) -> np.ndarray:
    """Visiting order of one sweep: array of (phase, i, j, k) rows."""
    lib = _load()
    T = num_triplets(n)
    rec = np.zeros((max(T, 1), 4), dtype=np.int32)
    cnt = lib.ora_order(n, schedule, tile,
                        rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), T)
    assert cnt == T, (cnt, T)
    return rec[:T]


def num_phases(n: int, schedule: int, tile: int = 16) -> int:
    return int(_load().ora_num_phases(n, schedule, tile))
