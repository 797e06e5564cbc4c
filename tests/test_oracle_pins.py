"""Pins for the oracle: each test checks the oracle against something other
than itself (the paper's worked case and counts, the defining property of a
projection, the invariant and dual ascent of Hildreth's method, a KKT
certificate, an exact LP solve, a closed-form optimum)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from instances import planted_partition, chung_lu, clustered

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_state(n, eps, seed, weights=True):
    d, w, _ = planted_partition(n, 2, 0.6, 0.3, seed, weights=(0.5, 2.0) if weights else None)
    return oracle.State(n, d, w, eps)


# ---- the worked triangle case of Sec. II-B ---------------------------------

def test_worked_triangle_case():
    g = json.load(open(os.path.join(GOLD, "worked_triangle.json")))
    for case in g["cases"]:
        for eps in (1.0, 0.2, 0.01):  # the projection step does not depend on eps
            s = oracle.State(3, np.zeros(3), np.ones(3), eps)
            s.x[:] = case["x_before"]  # packed order (0,1), (0,2), (1,2)
            s.visit_triplet(0, 1, 2, rows=1)
            np.testing.assert_allclose(s.x, case["x_after"], rtol=0, atol=2e-16)


# ---- one row is the W-weighted projection onto its halfspace ---------------

@pytest.mark.parametrize("seed", range(20))
def test_metric_row_is_weighted_projection(seed):
    rng = np.random.default_rng(seed)
    n = 4
    s = oracle.State(n, np.zeros(6), rng.uniform(0.3, 3.0, 6), 0.3)
    s.x[:] = rng.uniform(-1, 2, 6)
    if seed % 5 == 0:  # an exactly tight row: delta == 0
        s.x[oracle.pidx(n, 0, 1)] = s.x[oracle.pidx(n, 0, 2)] + s.x[oracle.pidx(n, 1, 2)]
    v = s.x.copy()
    i, j, k = 0, 1, 2
    s.visit_triplet(i, j, k, rows=1)   # y = 0, so this is a pure projection
    u = s.x.copy()
    a = np.zeros(6)
    a[oracle.pidx(n, i, j)] = 1
    a[oracle.pidx(n, i, k)] = -1
    a[oracle.pidx(n, j, k)] = -1
    W = s.w
    assert a @ u <= 1e-14                           # lands in the halfspace
    if a @ v <= 0:
        assert np.array_equal(u, v)                 # feasible points do not move
    # variational inequality of the W-projection onto {a.q <= 0}:
    # (v - u)^T W (q - u) <= 0 for every feasible q
    for _ in range(200):
        q = rng.uniform(-3, 3, 6)
        if a @ q > 0:
            q = q - (a @ q) / (a @ a) * a * rng.uniform(1.0, 2.0)
        assert a @ q <= 1e-12
        assert (v - u) @ (W * (q - u)) <= 1e-12
    # entries outside the row do not move
    other = a == 0
    assert np.array_equal(u[other], v[other])


@pytest.mark.parametrize("seed", range(10))
def test_pair_rows_are_weighted_projections(seed):
    rng = np.random.default_rng(100 + seed)
    s = oracle.State(2, np.array([float(seed % 2)]), np.array([rng.uniform(0.3, 3)]), 0.4)
    for row, a_row in ((1, np.array([1.0, -1.0])), (2, np.array([-1.0, -1.0]))):
        s.x[0], s.f[0] = rng.uniform(-2, 2), rng.uniform(-2, 2)
        s.ypair[:] = 0
        b = s.d[0] if row == 1 else -s.d[0]
        if row == 2:  # first row must be a no-op to isolate the second one
            s.x[0] = s.d[0] + s.f[0] - 0.5
        v = np.array([s.x[0], s.f[0]])
        s.visit_pair(0, rows=row)
        u = np.array([s.x[0], s.f[0]])
        assert a_row @ u <= b + 1e-14
        for _ in range(100):
            q = rng.uniform(-3, 3, 2)
            if a_row @ q > b:
                q = q - (a_row @ q - b) / 2.0 * a_row * rng.uniform(1.0, 2.0)
            assert (v - u) @ (s.w[0] * (q - u)) <= 1e-12


# ---- accumulated state: invariant and dual ascent --------------------------

@pytest.mark.parametrize("n,schedule,sweeps", [(5, 0, 1), (7, 1, 3), (9, 2, 2), (12, 1, 5), (12, 0, 4), (11, 2, 6)])
def test_invariant_v_equals_v0_minus_Winv_AT_y(n, schedule, sweeps):
    s = _rand_state(n, 0.25, seed=n + schedule)
    for _ in range(sweeps):
        s.sweep(schedule, tile=4)
    r = dense.invariant_residual(n, s.d, s.w, s.eps, s.x, s.f, s.ytri, s.ypair)
    assert r <= 1e-12
    assert s.ytri.min() >= 0 and s.ypair.min() >= 0


def test_invariant_mid_sweep():
    n = 8
    s = _rand_state(n, 0.5, seed=3)
    s.sweep(1)
    M = 3 * oracle.num_triplets(n) + 2 * oracle.num_pairs(n)
    for rows in (1, 2, 7, 50, M - 3, M - 1):
        t = s.copy()
        t.sweep(1, max_rows=rows)
        assert dense.invariant_residual(n, t.d, t.w, t.eps, t.x, t.f, t.ytri, t.ypair) <= 1e-12


@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_dual_objective_never_decreases(schedule):
    """Hildreth's method is exact coordinate ascent on the dual, so D(y)
    (computed from y alone through the dense matrix) never decreases."""
    n = 6
    s = _rand_state(n, 0.3, seed=11)
    M = 3 * oracle.num_triplets(n) + 2 * oracle.num_pairs(n)
    prev = dense.dual_objective(n, s.d, s.w, s.eps, s.ytri, s.ypair)
    base = s
    for _ in range(3):
        for rows in range(1, M + 1):
            t = base.copy()
            t.sweep(schedule, tile=4, max_rows=rows)
            D = dense.dual_objective(n, t.d, t.w, t.eps, t.ytri, t.ypair)
            assert D >= prev - 1e-12 * max(1.0, abs(prev))
            prev = D
        base.sweep(schedule, tile=4)


# ---- converged point -------------------------------------------------------

@pytest.mark.parametrize("n,schedule", [(6, 0), (8, 1), (10, 2)])
def test_kkt_certificate_at_convergence(n, schedule):
    s = _rand_state(n, 0.2, seed=n)
    assert s.solve(1e-11, 100000, schedule, tile=4) > 0
    k = dense.kkt(n, s.d, s.w, s.eps, s.x, s.f, s.ytri, s.ypair)
    assert k["primal"] <= 1e-9
    assert k["dual_neg"] == 0.0
    assert k["compl"] <= 1e-8
    assert k["stationarity"] <= 1e-10


@pytest.mark.parametrize("seed", range(3))
def test_lp_value_matches_highs_for_small_eps(seed):
    """Exact regularization (Sec. II-B): for eps small enough the QP solution
    solves the LP (mn1); compare the LP value with an exact HiGHS solve."""
    for n in (6, 8):
        d, w, _ = planted_partition(n, 2, 0.7, 0.2, seed, weights=(0.5, 2.0))
        lpv, _, _ = dense.lp_optimum(n, d, w)
        s = oracle.State(n, d, w, 0.02)
        assert s.solve(1e-12, 200000, schedule=1) > 0
        assert abs(s.objectives()["lp"] - lpv) <= 1e-6 * lpv


@pytest.mark.parametrize("n,k,eps", [(30, 3, 0.2), (41, 5, 1.0), (24, 2, 0.05)])
def test_closed_form_clustered_instance(n, k, eps):
    """For d the ultrametric of a clustering and eps <= 1 the QP optimum is
    x = d, f = 0 with pair duals y+ = w(1 - eps d)/2, y- = w(1 + eps d)/2."""
    d, w, _ = clustered(n, k, seed=n, weights=(0.5, 2.0))
    s = oracle.State(n, d, w, eps)
    assert s.solve(1e-13, 20000, schedule=1) > 0
    for _ in range(20):
        s.sweep(1)
    np.testing.assert_allclose(s.x, d, atol=1e-10)
    np.testing.assert_allclose(s.f, 0.0, atol=1e-10)
    np.testing.assert_allclose(s.ypair[0::2], w * (1 - eps * d) / 2, atol=1e-9)
    np.testing.assert_allclose(s.ypair[1::2], w * (1 + eps * d) / 2, atol=1e-9)
    assert s.ytri.max() <= 1e-9


# ---- derived quantities against their definitions -------------------------

@pytest.mark.parametrize("seed", range(5))
def test_violation_and_objectives_match_dense_definitions(seed):
    """The derived quantities are pure functions of the state: check them on
    arbitrary states (random x, f, y) against the dense rows."""
    n = 9
    s = _rand_state(n, 0.3, seed=5 + seed)
    rng = np.random.default_rng(seed)
    s.x[:] = rng.uniform(-0.5, 1.5, s.x.shape)
    s.f[:] = rng.uniform(-1.0, 1.0, s.f.shape)
    s.ytri[:] = rng.uniform(0, 1, s.ytri.shape)
    s.ypair[:] = rng.uniform(0, 1, s.ypair.shape)
    A, b = dense.constraint_matrix(n, s.d)
    v = np.concatenate([s.x, s.f])
    T3 = 3 * oracle.num_triplets(n)
    r = A @ v - b
    assert s.max_violation() == pytest.approx(max(0.0, r[:T3].max()), abs=1e-15)
    o = s.objectives()
    assert o["pair_violation"] == pytest.approx(max(0.0, r[T3:].max()), abs=1e-15)
    assert o["lp"] == pytest.approx(np.sum(s.w * np.abs(s.x - s.d)), rel=1e-14)
    assert o["qp_primal"] == pytest.approx(dense.qp_objective(s.d, s.w, s.eps, s.x, s.f), rel=1e-13)
    # on a state that satisfies the invariant (any iterate), the dual
    # objective from (x, f, y_pair) equals D(y) from the dense matrix
    t = _rand_state(n, 0.3, seed=5 + seed)
    t.sweep(1)
    t.sweep(2, tile=4, max_rows=100 + 17 * seed)
    D = dense.dual_objective(n, t.d, t.w, t.eps, t.ytri, t.ypair)
    assert t.objectives()["dual"] == pytest.approx(D, rel=1e-12)


def test_rank_and_pair_index_are_lexicographic():
    for n in (3, 4, 7, 13):
        for t, (i, j, k) in enumerate(itertools.combinations(range(n), 3)):
            assert oracle.trank(n, i, j, k) == t
        for t, (i, j) in enumerate(itertools.combinations(range(n), 2)):
            assert oracle.pidx(n, i, j) == t


def test_init_is_minus_inv_eps_W_inv_c():
    n = 7
    s = _rand_state(n, 0.37, seed=2)
    assert np.all(s.x == 0.0)
    assert np.all(s.f == -1.0 / 0.37)
    assert np.all(s.ytri == 0) and np.all(s.ypair == 0)
