"""Pins of the oracle's l2 metric nearness mode (Sec. II-A, Eq. metricnear with
p = 2, solved as Eq. qp with eps = 1, c = -W d by Algorithm 1 over the metric
rows only) against facts that do not come from the oracle: the closed-form
weighted projection onto one halfspace (n = 3), metric inputs that are their
own solution, the optimum from an active-set NNLS solve of the dual, KKT
conditions, and the dual objective evaluated directly from y."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import dense


def _solve(s, schedule=1, tile=4, viol=1e-13, gap=1e-12, max_sweeps=200000):
    """Sweep until the iterate is feasible and the duality gap has closed:
    Dykstra's iterate can be feasible long before it is optimal."""
    for k in range(1, max_sweeps + 1):
        s.sweep(schedule, tile)
        if s.max_violation() <= viol and abs(s.objectives()["gap"]) <= gap:
            return k
    return -1


pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.mark.parametrize("hyp", [0, 1, 2])
@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_single_triangle_is_the_weighted_halfspace_projection(hyp, schedule):
    # pairs of n = 3 in packed order: (0,1), (0,2), (1,2); row r of the
    # triplet has hypotenuse pair r (ij, ik, jk)
    w = np.array([0.7, 1.9, 1.3])
    d = np.array([0.2, 0.3, 0.25])
    d[hyp] = 1.4                                  # violates row `hyp` only
    legs = [p for p in range(3) if p != hyp]
    delta = d[hyp] - d[legs[0]] - d[legs[1]]
    awa = np.sum(1.0 / w)
    theta = delta / awa
    x_ref = d.copy()
    x_ref[hyp] -= theta / w[hyp]
    x_ref[legs] += theta / w[legs]
    s = oracle.State(3, d, w, problem="l2")
    for _ in range(3):                            # a fixed point after the first sweep
        s.sweep(schedule, 2)
        np.testing.assert_allclose(s.x, x_ref, rtol=1e-15, atol=1e-15)
        y = np.zeros(3)
        y[hyp] = theta
        np.testing.assert_allclose(s.ytri, y, rtol=1e-14, atol=1e-16)
    ob = s.objectives()
    assert ob["lp"] == pytest.approx(np.sum(w * (x_ref - d) ** 2), rel=1e-13)
    assert ob["gap"] == pytest.approx(0.0, abs=1e-14)


def test_a_metric_input_is_its_own_solution_bitwise():
    rng = np.random.default_rng(3)
    n = 14
    labels = rng.integers(0, 4, n)
    d = np.array([0.0 if labels[i] == labels[j] else 1.0 for i, j in itertools.combinations(range(n), 2)])
    w = rng.uniform(0.5, 2.0, len(d))
    s = oracle.State(n, d, w, problem="l2")
    for sched in (0, 1, 2):
        s.sweep(sched, 4)
    assert np.array_equal(s.x, d) and not s.ytri.any()
    assert s.max_violation() == 0.0 and s.objectives()["lp"] == 0.0


@pytest.mark.parametrize("n,weighted,seed", [(5, False, 0), (6, True, 1), (7, True, 2)])
def test_converged_oracle_matches_the_nnls_optimum(n, weighted, seed):
    rng = np.random.default_rng(seed)
    P = n * (n - 1) // 2
    d = rng.uniform(0.0, 1.0, P)
    w = rng.uniform(0.5, 2.0, P) if weighted else np.ones(P)
    x_ref, y_ref = dense.l2_optimum(n, d, w)
    assert dense.l2_kkt(n, d, w, x_ref, y_ref)["primal"] <= 1e-12     # the reference itself is optimal
    s = oracle.State(n, d, w, problem="l2")
    assert _solve(s) > 0
    np.testing.assert_allclose(s.x, x_ref, atol=1e-9)
    ob = s.objectives()
    assert ob["lp"] == pytest.approx(np.sum(w * (x_ref - d) ** 2), rel=1e-8)
    k = dense.l2_kkt(n, d, w, s.x, s.ytri)
    assert k["primal"] <= 1e-13 and k["dual_neg"] == 0.0
    assert k["compl"] <= 1e-10 and k["stationarity"] <= 1e-12
    assert abs(ob["gap"]) <= 1e-9


@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_dual_objective_through_the_invariant_equals_the_direct_one(schedule):
    rng = np.random.default_rng(4)
    n = 9
    P = n * (n - 1) // 2
    d = rng.uniform(0.0, 1.0, P)
    w = rng.uniform(0.5, 2.0, P)
    s = oracle.State(n, d, w, problem="l2")
    for _ in range(4):
        s.sweep(schedule, 4)
        ob = s.objectives()
        assert ob["dual"] == pytest.approx(dense.l2_dual_objective(n, d, w, s.ytri), rel=1e-12, abs=1e-13)
        # the identity Algorithm 1 keeps: W (x - d) = -A^T y
        A = dense.metric_matrix(n)
        assert np.max(np.abs(w * (s.x - d) + A.T @ s.ytri)) <= 1e-13


def test_schedules_reach_the_same_optimum():
    rng = np.random.default_rng(5)
    n = 8
    P = n * (n - 1) // 2
    d = rng.uniform(0.0, 1.0, P)
    w = np.ones(P)
    xs = []
    for sched in (0, 1, 2):
        s = oracle.State(n, d, w, problem="l2")
        assert _solve(s, schedule=sched) > 0
        xs.append(s.x.copy())
    np.testing.assert_allclose(xs[0], xs[1], atol=1e-9)
    np.testing.assert_allclose(xs[0], xs[2], atol=1e-9)


def test_worked_triangle_case_is_the_l2_solution():
    """The paper's worked projection (Sec. II-B, W = I, tests/golden/
    worked_triangle.json) is an l2 metric nearness step: starting from
    x = d = x_before, one l2 sweep of n = 3 gives x_after, which is then the
    optimum (one halfspace active)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_triangle.json")))
    for case in g["cases"]:
        d = np.array(case["x_before"])
        for sched in (0, 1, 2):
            s = oracle.State(3, d, np.ones(3), problem="l2")
            s.sweep(sched, 2)
            np.testing.assert_allclose(s.x, case["x_after"], rtol=0, atol=2e-16)
            s.sweep(sched, 2)
            np.testing.assert_allclose(s.x, case["x_after"], rtol=0, atol=2e-16)
