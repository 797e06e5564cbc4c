"""Seeded synthetic correlation-clustering instances.

This module only draws inputs; it holds none of the solver's arithmetic and is
shared by the tests, the oracle runs and the benchmark.  The paper builds its
instances from real graphs (Sec. IV-B); those are replaced here by synthetic
signed graphs of the same kind:

* pairs are numbered row-major over i<j (the packed order p(i,j));
* edge draws come first, from ``numpy.random.default_rng(seed)``, one uniform
  per pair in packed order; an edge exists when the draw is below p_ij;
* d_ij = 0 for an edge (a "positive" pair) and 1 otherwise (Sec. II-A);
* weights are 1, or uniform in [lo, hi] drawn from ``default_rng(seed + 1)``.
"""
from __future__ import annotations

import numpy as np


def _pairs(n: int):
    iu, ju = np.triu_indices(n, k=1)  # row-major i<j
    return iu, ju


def _finish(n, prob, seed, weights):
    rng = np.random.default_rng(seed)
    u = rng.random(prob.shape[0])
    edge = u < prob
    d = np.where(edge, 0.0, 1.0)
    P = prob.shape[0]
    if weights is None:
        w = np.ones(P)
    else:
        lo, hi = weights
        w = np.random.default_rng(seed + 1).uniform(lo, hi, P)
    return d, w, edge


def planted_partition(n: int, k: int, p_in: float, p_out: float, seed: int,
                      weights=None, labels=None):
    """Planted partition: node i in cluster i // ceil(n/k) unless ``labels``
    is given.  Returns (d, w, labels)."""
    if labels is None:
        size = -(-n // k)
        labels = np.arange(n) // size
    labels = np.asarray(labels)
    iu, ju = _pairs(n)
    prob = np.where(labels[iu] == labels[ju], p_in, p_out)
    d, w, _ = _finish(n, prob, seed, weights)
    return d, w, labels


def chung_lu(n: int, gamma: float, mean_degree: float, seed: int, weights=None):
    """Chung-Lu graph with power-law expected degrees:
    theta_i = c (i+1)^(-1/(gamma-1)) scaled so that mean(theta) = mean_degree,
    p_ij = min(1, theta_i theta_j / sum(theta)).  Returns (d, w, degrees)."""
    base = (np.arange(n) + 1.0) ** (-1.0 / (gamma - 1.0))
    theta = base * (mean_degree / base.mean())
    iu, ju = _pairs(n)
    prob = np.minimum(1.0, theta[iu] * theta[ju] / theta.sum())
    d, w, edge = _finish(n, prob, seed, weights)
    deg = np.bincount(iu[edge], minlength=n) + np.bincount(ju[edge], minlength=n)
    return d, w, deg


def clustered(n: int, k: int, seed: int = 0, weights=None):
    """Perfectly clusterable instance (p_in = 1, p_out = 0) with random
    cluster labels; d is then the cluster ultrametric."""
    labels = np.random.default_rng(seed).integers(0, k, n)
    d, w, _ = planted_partition(n, k, 1.0, 0.0, seed, weights=weights, labels=labels)
    return d, w, labels


def batch_planted(count: int, n_lo: int, n_hi: int, k_lo: int, k_hi: int,
                  p_in: float, p_out: float, seed: int):
    """Many planted-partition instances of uneven size: n ~ U[n_lo, n_hi],
    k ~ U[k_lo, k_hi], cluster ids uniform over k.  Returns a list of (n, d, w)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        k = int(rng.integers(k_lo, k_hi + 1))
        labels = rng.integers(0, k, n)
        d, w, _ = planted_partition(n, k, p_in, p_out, seed * 100003 + t, labels=labels)
        out.append((n, d, w))
    return out


def random_dissimilarity(n: int, seed: int, weights=None):
    """Dissimilarities d_ij ~ U[0, 1] drawn in packed order from
    default_rng(seed) (a classic metric nearness input: about a sixth of the
    metric rows start violated); weights as in _finish.  Returns (d, w)."""
    P = n * (n - 1) // 2
    d = np.random.default_rng(seed).random(P)
    w = np.ones(P) if weights is None else np.random.default_rng(seed + 1).uniform(weights[0], weights[1], P)
    return d, w


def noisy_euclidean(n: int, dim: int, noise: float, seed: int):
    """Distances of n points uniform in [0, 1]^dim, each multiplied by
    (1 + noise * u), u ~ U[-1, 1] (points first, then one u per pair in
    packed order, from default_rng(seed)); unit weights.  Returns (d, w)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, dim))
    iu, ju = _pairs(n)
    dist = np.sqrt(((pts[iu] - pts[ju]) ** 2).sum(1))
    d = dist * (1.0 + noise * rng.uniform(-1.0, 1.0, len(iu)))
    return d, np.ones(len(iu))


# Named workloads (sizes of the paper-shaped synthetic inputs).
def workload(name: str):
    """Return (n, d, w, description) for a named workload."""
    if name == "planted60":
        d, w, _ = planted_partition(60, 4, 0.8, 0.1, seed=0)
        return 60, d, w, "planted partition n=60, 4x15, p 0.8/0.1, seed 0, unit weights"
    if name == "chunglu1000":
        d, w, _ = chung_lu(1000, 2.5, 8.0, seed=1)
        return 1000, d, w, "Chung-Lu n=1000, exponent 2.5, mean degree 8, seed 1, unit weights"
    if name == "chunglu3000w":
        d, w, _ = chung_lu(3000, 2.5, 10.0, seed=2, weights=(0.5, 2.0))
        return 3000, d, w, "Chung-Lu n=3000, exponent 2.5, mean degree 10, seed 2, w~U[0.5,2]"
    if name == "chunglu1000perm":
        n = 1000
        d, w, _ = chung_lu(n, 2.5, 8.0, seed=1)
        perm = np.random.default_rng(7).permutation(n)
        D = np.zeros((n, n))
        iu, ju = np.triu_indices(n, 1)
        D[iu, ju] = d
        D = D + D.T
        Dp = D[np.ix_(perm, perm)]
        return n, Dp[iu, ju].copy(), w, "Chung-Lu n=1000 as chunglu1000 with node labels permuted (seed 7)"
    if name == "chunglu1000deal":
        n, B = 1000, 16
        d, w, _ = chung_lu(n, 2.5, 8.0, seed=1)
        nb = -(-n // B)
        sizes = [min(B, n - b * B) for b in range(nb)]
        label = np.empty(n, dtype=np.int64)     # original node -> new label, dealt round by round
        i = 0
        for r in range(B):
            for b in range(nb):
                if sizes[b] > r:
                    label[i] = b * B + r
                    i += 1
        order = np.argsort(label)               # new label -> original node
        D = np.zeros((n, n))
        iu, ju = np.triu_indices(n, 1)
        D[iu, ju] = d
        D = D + D.T
        Dp = D[np.ix_(order, order)]
        return n, Dp[iu, ju].copy(), w, "Chung-Lu n=1000 relabeled by dealing nodes over 16-blocks"
    if name.startswith("chunglu") and name[7:].isdigit():
        n = int(name[7:])
        d, w, _ = chung_lu(n, 2.5, 8.0, seed=1)
        return n, d, w, f"Chung-Lu n={n}, exponent 2.5, mean degree 8, seed 1, unit weights"
    raise KeyError(name)
