"""Brute-force checks from a dense constraint matrix (TEST INFRASTRUCTURE ONLY).

Builds the rows of Eq. (mn1) explicitly, independently of ``dykstra.c``:
pairs are numbered by enumerating ``itertools.combinations(range(n), 2)`` and
triplets by ``itertools.combinations(range(n), 3)`` (both lexicographic), so
no index formula is shared with the C code.  Rows: for every triplet the three
metric rows (hypotenuse ij, ik, jk), then for every pair the rows
x - f <= d and -x - f <= -d.  Columns: the x block, then the f block.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog


def pair_map(n: int) -> dict:
    return {pq: t for t, pq in enumerate(itertools.combinations(range(n), 2))}


def constraint_matrix(n: int, d: np.ndarray):
    """Sparse A (M x 2P) and b for the rows of Eq. (mn1)."""
    pm = pair_map(n)
    P = len(pm)
    rows, cols, vals, b = [], [], [], []
    r = 0
    for (i, j, k) in itertools.combinations(range(n), 3):
        ij, ik, jk = pm[(i, j)], pm[(i, k)], pm[(j, k)]
        for h, a1, a2 in ((ij, ik, jk), (ik, ij, jk), (jk, ij, ik)):
            rows += [r, r, r]
            cols += [h, a1, a2]
            vals += [1.0, -1.0, -1.0]
            b.append(0.0)
            r += 1
    for p in range(P):
        rows += [r, r]
        cols += [p, P + p]
        vals += [1.0, -1.0]
        b.append(d[p])
        r += 1
        rows += [r, r]
        cols += [p, P + p]
        vals += [-1.0, -1.0]
        b.append(-d[p])
        r += 1
    A = sp.csr_matrix((vals, (rows, cols)), shape=(r, 2 * P))
    return A, np.array(b)


def stack_duals(ytri: np.ndarray, ypair: np.ndarray) -> np.ndarray:
    """Dual vector in the row order of ``constraint_matrix``."""
    return np.concatenate([ytri, ypair])


def lp_optimum(n: int, d: np.ndarray, w: np.ndarray):
    """Solve the LP (mn1) exactly with HiGHS; returns (value, x, f)."""
    A, b = constraint_matrix(n, d)
    P = len(d)
    c = np.concatenate([np.zeros(P), w])
    res = linprog(c, A_ub=A, b_ub=b, bounds=[(None, None)] * (2 * P), method="highs")
    assert res.status == 0, res.message
    return res.fun, res.x[:P], res.x[P:]


def invariant_residual(n, d, w, eps, x, f, ytri, ypair) -> float:
    """max | v - (v0 - W^{-1} A^T y / eps) | with v0 = -(1/eps) W^{-1} c."""
    A, _ = constraint_matrix(n, d)
    P = len(d)
    winv = np.concatenate([1.0 / w, 1.0 / w])
    c = np.concatenate([np.zeros(P), w])
    y = stack_duals(ytri, ypair)
    v0 = -(1.0 / eps) * winv * c
    v = np.concatenate([x, f])
    return float(np.max(np.abs(v - (v0 - winv * (A.T @ y) / eps))))


def kkt(n, d, w, eps, x, f, ytri, ypair) -> dict:
    """KKT residuals of the QP (Eq. qp) at (v, y)."""
    A, b = constraint_matrix(n, d)
    P = len(d)
    v = np.concatenate([x, f])
    y = stack_duals(ytri, ypair)
    c = np.concatenate([np.zeros(P), w])
    W = np.concatenate([w, w])
    slack = b - A @ v
    return {
        "primal": float(max(0.0, -slack.min())),
        "dual_neg": float(max(0.0, -y.min())),
        "compl": float(np.max(np.abs(y * slack))),
        "stationarity": float(np.max(np.abs(c + eps * W * v + A.T @ y))),
    }


def qp_objective(d, w, eps, x, f) -> float:
    return float(np.sum(w * f) + 0.5 * eps * np.sum(w * (x * x + f * f)))


def dual_objective(n, d, w, eps, ytri, ypair) -> float:
    """D(y) = -b^T y - (1/(2 eps)) (c + A^T y)^T W^{-1} (c + A^T y), computed
    from the dense matrix (does not use the primal iterate)."""
    A, b = constraint_matrix(n, d)
    P = len(d)
    y = stack_duals(ytri, ypair)
    c = np.concatenate([np.zeros(P), w])
    winv = np.concatenate([1.0 / w, 1.0 / w])
    g = c + A.T @ y
    return float(-b @ y - 0.5 / eps * np.sum(winv * g * g))


# ---- l2 metric nearness (Eq. metricnear, p = 2) -------------------------------

def metric_matrix(n: int):
    """Sparse A (3T x P) of the metric rows alone, rows in the order of
    ``constraint_matrix`` (hypotenuse ij, ik, jk per triplet)."""
    pm = pair_map(n)
    rows, cols, vals = [], [], []
    r = 0
    for (i, j, k) in itertools.combinations(range(n), 3):
        ij, ik, jk = pm[(i, j)], pm[(i, k)], pm[(j, k)]
        for h, a1, a2 in ((ij, ik, jk), (ik, ij, jk), (jk, ij, ik)):
            rows += [r, r, r]
            cols += [h, a1, a2]
            vals += [1.0, -1.0, -1.0]
            r += 1
    return sp.csr_matrix((vals, (rows, cols)), shape=(r, len(pm)))


def l2_optimum(n: int, d: np.ndarray, w: np.ndarray):
    """min sum w (x - d)^2 s.t. the metric rows, through its dual: with
    M = W^{-1/2} A^T and q = W^{1/2} d the dual is min_{y >= 0} ||M y - q||,
    a non-negative least-squares problem (scipy's active-set NNLS); the
    unique primal solution is x = d - W^{-1} A^T y.  Returns (x, y)."""
    from scipy.optimize import nnls
    A = metric_matrix(n).toarray()
    M = (A / np.sqrt(w)[None, :]).T
    y, _ = nnls(M, np.sqrt(w) * d, maxiter=50 * A.shape[0])
    x = d - (A.T @ y) / w
    return x, y


def l2_kkt(n: int, d: np.ndarray, w: np.ndarray, x: np.ndarray, ytri: np.ndarray) -> dict:
    """KKT residuals of min (1/2) sum w (x - d)^2 s.t. A x <= 0 at (x, y)."""
    A = metric_matrix(n)
    ax = A @ x
    return {"primal": float(max(0.0, ax.max())), "dual_neg": float(max(0.0, -ytri.min())),
            "compl": float(np.max(np.abs(ytri * ax))),
            "stationarity": float(np.max(np.abs(w * (x - d) + A.T @ ytri)))}


def l2_dual_objective(n: int, d: np.ndarray, w: np.ndarray, ytri: np.ndarray) -> float:
    """y^T A d - (1/2) y^T A W^{-1} A^T y, evaluated from y directly."""
    A = metric_matrix(n)
    aty = A.T @ ytri
    return float(ytri @ (A @ d) - 0.5 * np.sum(aty * aty / w))
