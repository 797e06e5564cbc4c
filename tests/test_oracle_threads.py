"""The oracle's threaded sweep (units of a phase dealt to host threads, a
barrier at every phase end) against its serial sweep: the units of a phase
are disjoint (Sec. III-A, III-C), so every row sees the values it sees in the
serial walk and the two agree bit for bit, for every schedule, thread count
and partial sweep."""
import numpy as np
import pytest

import oracle
from instances import chung_lu, planted_partition, random_dissimilarity


def _state(problem, n, seed):
    if problem == "l2":
        d, w = random_dissimilarity(n, seed, weights=(0.5, 2.0))
        return oracle.State(n, d, w, problem="l2")
    d, w, _ = chung_lu(n, 2.5, 4.0, seed=seed, weights=(0.5, 2.0))
    return oracle.State(n, d, w, 0.2)


def _same(a, b):
    for k in ("x", "f", "ytri", "ypair"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)


@pytest.mark.parametrize("problem", ["cc", "l2"])
@pytest.mark.parametrize("schedule,tile", [(0, 16), (1, 16), (2, 4), (2, 8), (2, 16)])
@pytest.mark.parametrize("n", [3, 17, 41])
@pytest.mark.parametrize("threads", [1, 2, 3, 7, 16])
def test_threaded_sweeps_equal_serial_sweeps(problem, schedule, tile, n, threads):
    a = _state(problem, n, n + threads)
    b = a.copy()
    T, P = oracle.num_triplets(n), oracle.num_pairs(n)
    for _ in range(3):
        ra = a.sweep(schedule, tile)
        rb = b.sweep_threads(schedule, tile, threads)
        assert ra == rb == 3 * T + (2 * P if problem == "cc" else 0)
    _same(a, b)
    assert a.max_violation() == b.max_violation()


@pytest.mark.parametrize("schedule,tile", [(0, 16), (1, 16), (2, 8)])
@pytest.mark.parametrize("phases", [1, 2, 5])
def test_partial_sweep_is_the_first_phases(schedule, tile, phases):
    """max_phases = q visits exactly the metric rows of phases 0..q-1 in
    schedule order (checked against single-triplet visits), no pair rows."""
    n = 30
    a = _state("cc", n, 3)
    a.sweep(schedule, tile)                 # a state with nonzero duals
    b = a.copy()
    rec = oracle.order(n, schedule, tile)
    first = rec[rec[:, 0] < phases]
    for _, i, j, k in first:
        a.visit_triplet(int(i), int(j), int(k))
    rows = b.sweep_threads(schedule, tile, 4, max_phases=phases)
    assert rows == 3 * len(first)
    _same(a, b)


def test_more_threads_than_units():
    n = 6
    a = _state("cc", n, 1)
    b = a.copy()
    for _ in range(4):
        a.sweep(2, 4)
        b.sweep_threads(2, 4, 64)
    _same(a, b)


def test_threaded_solve_reaches_the_serial_result():
    n = 24
    d, w, _ = planted_partition(n, 3, 0.8, 0.1, seed=2)
    a = oracle.State(n, d, w, 0.2)
    b = a.copy()
    for _ in range(40):
        a.sweep(1)
        b.sweep_threads(1, threads=5)
    _same(a, b)
    assert a.objectives() == b.objectives()


@pytest.mark.parametrize("n", [3, 4, 23, 64])
@pytest.mark.parametrize("threads", [1, 2, 5, 16])
def test_threaded_max_violation_equals_serial(n, threads):
    """The threaded largest violation (first indices dealt to threads) is the
    serial one, exactly: a maximum does not depend on the order."""
    rng = np.random.default_rng(n * 31 + threads)
    x = rng.uniform(0.0, 1.0, oracle.num_pairs(n))
    serial = oracle.max_violation(n, x)
    assert oracle.max_violation(n, x, threads=threads) == serial
    st = oracle.State(n, np.ones(oracle.num_pairs(n)), np.ones(oracle.num_pairs(n)), 0.2)
    st.x[:] = x
    assert st.max_violation() == serial
