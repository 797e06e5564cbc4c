"""The seeded input recipe (instances/): determinism, packed pair order,
edge statistics of the planted-partition and Chung-Lu graphs, the weight
ranges, and the closed facts of the metric-nearness inputs (a sixth of the
rows of U[0,1] dissimilarities start violated; noise-free Euclidean
distances are a metric)."""
import itertools

import numpy as np
import pytest

from instances import (batch_planted, chung_lu, clustered, noisy_euclidean, planted_partition,
                       random_dissimilarity, workload)


def _violated_fraction(n, d):
    D = np.zeros((n, n))
    iu, ju = np.triu_indices(n, 1)
    D[iu, ju] = d
    D = D + D.T
    bad = tot = 0
    for i, j, k in itertools.combinations(range(n), 3):
        a, b, c = D[i, j], D[i, k], D[j, k]
        bad += (a > b + c) + (b > a + c) + (c > a + b)
        tot += 3
    return bad / tot


def test_generators_are_deterministic_and_packed_row_major():
    for make in (lambda s: planted_partition(40, 3, 0.7, 0.1, seed=s)[:2],
                 lambda s: chung_lu(50, 2.5, 6.0, seed=s, weights=(0.5, 2.0))[:2],
                 lambda s: random_dissimilarity(30, s), lambda s: noisy_euclidean(30, 2, 0.2, s)):
        a, b, c = make(3), make(3), make(4)
        assert all(np.array_equal(u, v) for u, v in zip(a, b))
        assert not np.array_equal(a[0], c[0])
    # packed order p(i, j) = i n - i(i+1)/2 + (j - i - 1): clusters {0..9}, {10..19}
    d, _, labels = planted_partition(20, 2, 1.0, 0.0, seed=0)
    n = 20
    for i, j in itertools.combinations(range(n), 2):
        p = i * n - i * (i + 1) // 2 + (j - i - 1)
        assert d[p] == (0.0 if labels[i] == labels[j] else 1.0)


def test_planted_partition_edge_rates():
    n, k = 400, 4
    d, w, labels = planted_partition(n, k, 0.7, 0.05, seed=5)
    iu, ju = np.triu_indices(n, 1)
    same = labels[iu] == labels[ju]
    assert set(np.unique(d)) <= {0.0, 1.0} and np.all(w == 1.0)
    assert abs((d[same] == 0).mean() - 0.7) < 0.02
    assert abs((d[~same] == 0).mean() - 0.05) < 0.01
    assert np.array_equal(labels, np.arange(n) // (n // k))


def test_chung_lu_degrees():
    n, mean = 2000, 8.0
    d, w, _ = chung_lu(n, 2.5, mean, seed=1, weights=(0.5, 2.0))
    iu, ju = np.triu_indices(n, 1)
    deg = np.bincount(iu[d == 0], minlength=n) + np.bincount(ju[d == 0], minlength=n)
    assert abs(deg.mean() - mean) < 0.1 * mean          # clipping at p = 1 only lowers it slightly
    assert deg[:20].mean() > 5 * deg[-200:].mean()      # expected degrees fall with the index
    assert w.min() >= 0.5 and w.max() <= 2.0 and abs(w.mean() - 1.25) < 0.01


def test_uniform_dissimilarities_violate_a_sixth_of_the_rows():
    n = 60
    d, w = random_dissimilarity(n, 9)
    assert d.min() >= 0.0 and d.max() < 1.0 and np.all(w == 1.0)
    assert abs(_violated_fraction(n, d) - 1.0 / 6.0) < 0.01   # P(X > Y + Z) = 1/6 for iid U[0,1]


def test_noise_free_euclidean_distances_are_a_metric():
    n = 40
    d, _ = noisy_euclidean(n, 3, 0.0, 2)
    D = np.zeros((n, n))
    iu, ju = np.triu_indices(n, 1)
    D[iu, ju] = d
    D = D + D.T
    for i, j, k in itertools.combinations(range(n), 3):
        assert D[i, j] <= D[i, k] + D[j, k] + 1e-12
    d2, _ = noisy_euclidean(n, 3, 0.5, 2)
    assert _violated_fraction(n, d2) > 0


def test_clustered_and_batch_instances():
    d, w, labels = clustered(30, 3, seed=1)
    iu, ju = np.triu_indices(30, 1)
    assert np.array_equal(d, np.where(labels[iu] == labels[ju], 0.0, 1.0))
    inst = batch_planted(12, 50, 80, 2, 5, 0.7, 0.05, seed=3)
    assert len(inst) == 12
    for n, d, w in inst:
        assert 50 <= n <= 80 and d.shape == w.shape == (n * (n - 1) // 2,)
    assert all(np.array_equal(a[1], b[1]) for a, b in zip(inst, batch_planted(12, 50, 80, 2, 5, 0.7, 0.05, seed=3)))


@pytest.mark.parametrize("name,n,weighted", [("planted60", 60, False), ("chunglu1000", 1000, False),
                                             ("chunglu1000perm", 1000, False)])
def test_named_workloads(name, n, weighted):
    m, d, w, desc = workload(name)
    assert m == n and d.shape == w.shape == (n * (n - 1) // 2,) and desc
    assert np.all(w == 1.0) != weighted


def test_permuted_workload_is_the_same_graph_relabeled():
    n, d, _, _ = workload("chunglu1000")
    _, dp, _, _ = workload("chunglu1000perm")
    iu, ju = np.triu_indices(n, 1)
    deg = lambda x: np.sort(np.bincount(iu[x == 0], minlength=n) + np.bincount(ju[x == 0], minlength=n))
    assert (d == 0).sum() == (dp == 0).sum() and np.array_equal(deg(d), deg(dp))
    assert not np.array_equal(d, dp)
