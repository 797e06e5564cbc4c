"""GPU path against the oracle on the same seeded inputs (through the C ABI).

Tolerances: the exact mode evaluates every row operation by operation in
IEEE double in the oracle's rounding order, so it must agree bit for bit.
The fused form differs from the oracle only in rounding: one sweep from an
identical state must agree to 1e-12 in the norm
||gpu - oracle||_inf / max(||oracle||_inf, 1) on x, f and y; at convergence
the LP objective must agree to 1e-6 relative and the violation be <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from instances import planted_partition, chung_lu, clustered, workload

pytestmark = pytest.mark.gpu

TOL_SWEEP = 1e-12


def _solver(n, d, w, **kw):
    """Tiled schedule on consecutive blocks (no relabeling), the order the
    oracle's schedule 2 walks; the relabeled order is tested separately."""
    import paper_1901_10084_gb300 as cc
    kw.setdefault("interleave", False)
    return cc.Solver(n, d, w, **kw)


def _gpu_state(s):
    x, f = s.get_x()
    yt, yp = s.get_duals()
    return x, f, yt, yp


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0)) if a.size else 0.0


def _assert_state_close(g, o, tol):
    x, f, yt, yp = g
    assert _rel(x, o.x) <= tol
    assert _rel(f, o.f) <= tol
    assert _rel(yt, o.ytri) <= tol
    assert _rel(yp, o.ypair) <= tol


def _assert_state_equal(g, o):
    x, f, yt, yp = g
    np.testing.assert_array_equal(x, o.x)
    np.testing.assert_array_equal(f, o.f)
    np.testing.assert_array_equal(yt, o.ytri)
    np.testing.assert_array_equal(yp, o.ypair)


# ---------------------------------------------------------------- exact mode

@pytest.mark.parametrize("n,tile,weighted", [(60, 16, False), (60, 8, True), (61, 16, True),
                                             (37, 32, False), (3, 8, False), (17, 16, True),
                                             (100, 8, False)])
def test_exact_mode_is_bitwise_equal(n, tile, weighted):
    d, w, _ = planted_partition(n, 4, 0.8, 0.1, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    with _solver(n, d, w, eps=0.2, tile=tile, exact=True) as s:
        o.sweep(2, tile)
        s.sweep(1)
        _assert_state_equal(_gpu_state(s), o)
        o.sweep(2, tile)
        o.sweep(2, tile)
        s.sweep(2)
        _assert_state_equal(_gpu_state(s), o)


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("n,weighted", [(60, False), (61, True), (3, False), (4, True), (33, False)])
def test_paper_schedules_exact_bitwise(schedule, n, weighted):
    """Schedules 0 (the paper's diagonal schedule) and 1 (sum mod n) on the
    GPU, row by row as Algorithm 1 states it: bit-identical to the oracle."""
    d, w, _ = planted_partition(n, 3, 0.8, 0.1, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    with _solver(n, d, w, eps=0.2, schedule=schedule, exact=True) as s:
        o.sweep(schedule)
        s.sweep(1)
        _assert_state_equal(_gpu_state(s), o)
        o.sweep(schedule)
        o.sweep(schedule)
        s.sweep(2)
        _assert_state_equal(_gpu_state(s), o)
        assert s.check()["max_violation"] == o.max_violation()


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("n,weighted", [(80, True), (150, False)])
def test_paper_schedules_fused_one_sweep(schedule, n, weighted):
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    for _ in range(3):
        o.sweep(schedule)
    with _solver(n, d, w, eps=0.2, schedule=schedule) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        s.sweep(1)
        o.sweep(schedule)
        _assert_state_close(_gpu_state(s), o, TOL_SWEEP)
        T = n * (n - 1) * (n - 2) // 6
        full, _ = s.get_duals()
        part, _ = s.get_duals(T // 3, 500, pairs=False)
        np.testing.assert_array_equal(part, full[3 * (T // 3): 3 * (T // 3 + 500)])


@pytest.mark.parametrize("schedule", [0, 1])
def test_paper_schedules_converge_planted60(schedule):
    n, d, w, _ = workload("planted60")
    o = oracle.State(n, d, w, 0.2)
    ko = o.solve(1e-4, 5000, schedule=schedule, check_every=1)
    with _solver(n, d, w, eps=0.2, schedule=schedule, check_every=1) as s:
        conv, kg = s.solve(1e-4, 5000)
        st = s.check()
    assert conv and kg == ko
    assert abs(st["lp_objective"] - o.objectives()["lp"]) <= 1e-6 * o.objectives()["lp"]


# ---------------------------------------------------------------- fused form

@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("n,tile,weighted,pre", [(60, 16, False, 3), (61, 16, True, 5),
                                                 (200, 16, False, 2), (150, 8, True, 2),
                                                 (90, 8, True, 4), (203, 8, False, 6)])
def test_fused_one_sweep_from_identical_state(n, tile, weighted, pre, variant):
    """variant 1: one CTA per block triple; 2: one warp; 3: a half-size CTA."""
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    for _ in range(pre):
        o.sweep(2, tile)
    with _solver(n, d, w, eps=0.2, tile=tile, variant=variant) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        _assert_state_close(_gpu_state(s), o, 1e-15)   # round trip of the state
        s.sweep(1)
        o.sweep(2, tile)
        _assert_state_close(_gpu_state(s), o, TOL_SWEEP)


def _line_metric_state(n, seed, noise):
    """x_ij = |p_i - p_j| for points on a line (every triplet has one row that
    is tight up to rounding), plus noise of the given sizes on some pairs: rows
    sit on both sides of zero, close to the float pre-filter's threshold."""
    rng = np.random.default_rng(seed)
    p = np.sort(rng.uniform(0, 1, n))
    iu, ju = np.triu_indices(n, 1)
    x = np.abs(p[iu] - p[ju])
    sizes = rng.choice(noise, size=x.shape)
    x = x + sizes * rng.choice([-1.0, 0.0, 1.0], size=x.shape)
    return x


@pytest.mark.parametrize("n,tile,weighted", [(40, 8, False), (70, 16, True), (90, 32, False)])
def test_fused_near_tight_rows(n, tile, weighted):
    """Rows with delta within a few float ulps of zero must not be skipped
    wrongly: one fused sweep from such a state matches the oracle."""
    d, w, _ = planted_partition(n, 3, 0.7, 0.2, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    o.x[:] = _line_metric_state(n, n, [1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 0.0])
    o.f[:] = 0.05
    with _solver(n, d, w, eps=0.2, tile=tile) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        st = s.check()
        assert st["max_violation"] == o.max_violation()
        s.sweep(1)
        o.sweep(2, tile)
        _assert_state_close(_gpu_state(s), o, TOL_SWEEP)
        st = s.check()      # x now differs from the oracle's by rounding only
        assert st["max_violation"] == pytest.approx(o.max_violation(), abs=1e-12)


@pytest.mark.parametrize("n,tile,weighted", [(150, 32, True), (97, 32, False)])
def test_fused_tile32_cta_kernel(n, tile, weighted):
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    for _ in range(2):
        o.sweep(2, tile)
    with _solver(n, d, w, eps=0.2, tile=tile) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        s.sweep(2)
        o.sweep(2, tile)
        o.sweep(2, tile)
        _assert_state_close(_gpu_state(s), o, 2 * TOL_SWEEP)


def test_fused_matches_over_many_sweeps_planted60():
    n, d, w, _ = workload("planted60")
    o = oracle.State(n, d, w, 0.2)
    with _solver(n, d, w, eps=0.2, tile=16) as s:
        for _ in range(20):
            o.sweep(2, 16)
        s.sweep(20)
        # errors of the fused form stay at rounding level over many sweeps
        _assert_state_close(_gpu_state(s), o, 1e-11)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_converged_objective_planted60(tile):
    n, d, w, _ = workload("planted60")
    o = oracle.State(n, d, w, 0.2)
    ko = o.solve(1e-4, 5000, schedule=2, tile=tile, check_every=1)
    assert ko > 0
    with _solver(n, d, w, eps=0.2, tile=tile, check_every=1) as s:
        conv, kg = s.solve(1e-4, 5000)
        st = s.check()
    assert conv and st["max_violation"] <= 1e-4
    assert kg == ko
    oo = o.objectives()
    assert abs(st["lp_objective"] - oo["lp"]) <= 1e-6 * abs(oo["lp"])
    assert abs(st["qp_primal"] - oo["qp_primal"]) <= 1e-6 * abs(oo["qp_primal"])


def test_check_quantities_match_oracle():
    n = 70
    d, w, _ = planted_partition(n, 3, 0.7, 0.2, seed=4, weights=(0.5, 2.0))
    o = oracle.State(n, d, w, 0.3)
    for _ in range(4):
        o.sweep(2, 16)
    with _solver(n, d, w, eps=0.3, tile=16, exact=True) as s:
        s.sweep(4)
        st = s.check()
    oo = o.objectives()
    assert st["max_violation"] == o.max_violation()        # same x, same arithmetic
    assert st["pair_violation"] == pytest.approx(oo["pair_violation"], abs=1e-15)
    for k_gpu, k_ora in (("lp_objective", "lp"), ("qp_primal", "qp_primal"), ("dual_objective", "dual"),
                         ("wf", "wf")):
        assert st[k_gpu] == pytest.approx(oo[k_ora], rel=1e-12, abs=1e-12)


def test_dual_range_queries():
    n = 45
    d, w, _ = planted_partition(n, 3, 0.7, 0.2, seed=2)
    with _solver(n, d, w, tile=8) as s:
        s.sweep(3)
        full, yp = s.get_duals()
        T = n * (n - 1) * (n - 2) // 6
        for first, count in ((0, 1), (5, 100), (T - 7, 7), (1234, 3000), (0, 0)):
            part, _ = s.get_duals(first, count, pairs=False)
            np.testing.assert_array_equal(part, full[3 * first: 3 * (first + count)])


def test_resume_is_exact():
    """run(k1 + k2) == run(k1); save; restore into a new handle; run(k2)."""
    n = 50
    d, w, _ = planted_partition(n, 3, 0.7, 0.2, seed=9, weights=(0.5, 2.0))
    with _solver(n, d, w, tile=16, exact=True) as a:
        a.sweep(7)
        ref = _gpu_state(a)
    with _solver(n, d, w, tile=16, exact=True) as b:
        b.sweep(4)
        snap = _gpu_state(b)
    with _solver(n, d, w, tile=16, exact=True) as c:
        c.set_state(*snap)
        c.sweep(3)
        got = _gpu_state(c)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


@pytest.mark.parametrize("n,k,eps", [(300, 6, 0.2), (130, 3, 1.0), (1000, 10, 0.2)])
def test_closed_form_clustered_on_gpu(n, k, eps):
    d, w, _ = clustered(n, k, seed=1, weights=(0.5, 2.0))
    with _solver(n, d, w, eps=eps, tile=16, check_every=5) as s:
        conv, _ = s.solve(1e-13, 5000)
        s.sweep(10)
        x, f = s.get_x()
        yt, yp = s.get_duals()
    assert conv
    np.testing.assert_allclose(x, d, atol=1e-10)
    np.testing.assert_allclose(f, 0.0, atol=1e-10)
    np.testing.assert_allclose(yp[0::2], w * (1 - eps * d) / 2, atol=1e-9)
    np.testing.assert_allclose(yp[1::2], w * (1 + eps * d) / 2, atol=1e-9)
    assert yt.max() <= 1e-9


def test_invalid_inputs_are_rejected():
    import paper_1901_10084_gb300 as cc
    n = 10
    P = n * (n - 1) // 2
    d, w = np.zeros(P), np.ones(P)
    bad_w = w.copy()
    bad_w[3] = 0.0
    with pytest.raises(cc.CCError) as e:
        cc.Solver(n, d, bad_w)
    assert e.value.code == cc.CC_ERR_ARG
    bad_d = d.copy()
    bad_d[7] = np.nan
    with pytest.raises(cc.CCError) as e:
        cc.Solver(n, bad_d, w)
    assert e.value.code == cc.CC_ERR_ARG


def test_barrier_time_limit_reports_and_context_survives():
    """One CTA leaves without arriving at the first barrier: the others hit
    the time limit, the sweep returns, the next check reports
    CC_ERR_TIMEOUT, and the context keeps working."""
    import paper_1901_10084_gb300 as cc
    n = 200
    d, w, _ = planted_partition(n, 4, 0.8, 0.1, seed=0)
    with _solver(n, d, w, tile=16, barrier_timeout_s=0.05, debug_skip_cta=0, grid=8) as s:
        s.sweep(1)
        with pytest.raises(cc.CCError) as e:
            s.check()
        assert e.value.code == cc.CC_ERR_TIMEOUT
    o = oracle.State(n, d, w, 0.2)
    o.sweep(2, 16)
    with _solver(n, d, w, tile=16, exact=True) as s:
        s.sweep(1)
        _assert_state_equal(_gpu_state(s), o)


@pytest.mark.parametrize("n,tile,weighted", [(300, 16, True), (217, 8, False)])
def test_one_sweep_late_in_the_solve(n, tile, weighted):
    """One GPU sweep from an oracle state 60 sweeps into the solve, where most
    rows carry nonzero duals and the row-skip filters decide differently than
    in the first sweeps: x, f and all duals within 1e-12 per sweep."""
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n + 3, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    for _ in range(60):
        o.sweep(2, tile)
    assert np.count_nonzero(o.ytri) > 1000
    with _solver(n, d, w, eps=0.2, tile=tile) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        s.sweep(1)
        o.sweep(2, tile)
        _assert_state_close(_gpu_state(s), o, TOL_SWEEP)


# ---------------------------------------------------------------- full size

def _caller_triplets(n, first, count):
    """Caller triplets i<j<k of lexicographic ranks [first, first + count)."""
    import itertools
    i = 0
    while oracle.trank(n, i + 1, i + 2, i + 3) <= first if i + 3 < n else False:
        i += 1
    out = []
    for t in itertools.combinations(range(i, n), 3):
        r = oracle.trank(n, *t)
        if r >= first + count:
            break
        if r >= first:
            out.append(t)
    assert len(out) == count
    return out


def test_full_size_chunglu1000_bench_configuration():
    """The benchmark workload in the launch configuration bench.py times
    (tile 16, relabeled objects, default sweep form): three sweeps from the
    start against the oracle run on the relabeled instance (the first sweep
    only moves the pair rows; the second and third have many active rows);
    x and f in full, the duals on three sampled ranges, mapped by hand."""
    from relabel import deal_labels
    n, d, w, _ = workload("chunglu1000")
    B = 16
    lab = deal_labels(n, B)
    iu, ju = np.triu_indices(n, 1)
    a, b = lab[iu], lab[ju]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    pmap = lo * n - lo * (lo + 1) // 2 + (hi - lo - 1)       # caller pair -> internal pair
    dint, wint = np.empty_like(d), np.empty_like(w)
    dint[pmap], wint[pmap] = d, w
    o = oracle.State(n, dint, wint, 0.2)
    with _solver(n, d, w, eps=0.2, tile=B, interleave=True) as s:
        for k in range(3):
            o.sweep(2, B)
            s.sweep(1)
        x, f = s.get_x()
        assert _rel(x, o.x[pmap]) <= TOL_SWEEP and _rel(f, o.f[pmap]) <= TOL_SWEEP
        T = n * (n - 1) * (n - 2) // 6
        for first in (0, T // 2, T - 40000):
            yt, _ = s.get_duals(first, 40000, pairs=False)
            ref = np.empty(3 * 40000)
            for q, (i, j, k) in enumerate(_caller_triplets(n, first, 40000)):
                li, lj, lk = lab[i], lab[j], lab[k]
                u, z = min(li, lj, lk), max(li, lj, lk)
                v = li + lj + lk - u - z
                base = 3 * oracle.trank(n, u, v, z)
                for row, out in enumerate((lk, lj, li)):      # caller row ij leaves k out, ik j, jk i
                    ref[3 * q + row] = o.ytri[base + (0 if out == z else 1 if out == v else 2)]
            assert _rel(yt, ref) <= TOL_SWEEP
        st = s.check()
    assert st["max_violation"] == pytest.approx(o.max_violation(), abs=1e-12)


def test_full_size_chunglu1000_exact_two_sweeps():
    """The exact form at full size, two sweeps from the start (the second with
    active rows): bit-identical to the oracle."""
    n, d, w, _ = workload("chunglu1000")
    o = oracle.State(n, d, w, 0.2)
    o.sweep(2, 16)
    o.sweep(2, 16)
    with _solver(n, d, w, eps=0.2, tile=16, exact=True) as s:
        s.sweep(2)
        x, f = s.get_x()
        assert np.array_equal(x, o.x) and np.array_equal(f, o.f)
        T = n * (n - 1) * (n - 2) // 6
        for first in (0, T // 2, T - 200000):
            yt, _ = s.get_duals(first, 200000, pairs=False)
            assert np.array_equal(yt, o.ytri[3 * first: 3 * (first + 200000)])


def test_random_configurations_track_the_oracle():
    """Seeded fuzzing against the oracle: random problem (CC LP or l2),
    schedule, form, tile, size (tiny and ragged included) and weights; a few
    sweeps from the start.  The exact form must equal the oracle bit for bit,
    the fused form stay within 1e-11 (a few sweeps of 1e-12 rounding)."""
    from instances import random_dissimilarity
    rng = np.random.default_rng(77)
    for case in range(20):
        problem = "l2" if rng.random() < 0.35 else "cc"
        schedule = int(rng.choice([0, 1, 2, 2]))
        exact = bool(rng.random() < 0.5)
        n = int(rng.choice([3, 4, 9, 20, 33, 48, 61, 80]))
        tile = int(rng.choice([8, 16, 32]))
        weighted = bool(rng.random() < 0.5)
        sweeps = int(rng.integers(1, 5))
        seed = int(rng.integers(0, 10**6))
        if problem == "l2":
            d, w = random_dissimilarity(n, seed, weights=(0.5, 2.0) if weighted else None)
            o = oracle.State(n, d, w, problem="l2")
        else:
            d, w, _ = chung_lu(n, 2.5, 8.0, seed=seed, weights=(0.5, 2.0) if weighted else None)
            o = oracle.State(n, d, w, 0.2)
        with _solver(n, d, w, eps=0.2, schedule=schedule, tile=tile, exact=exact, problem=problem) as s:
            s.sweep(sweeps)
            for _ in range(sweeps):
                o.sweep(schedule, tile)
            g = _gpu_state(s)
        what = (case, problem, schedule, exact, n, tile, weighted, sweeps)
        if exact:
            for u, v in zip(g, (o.x, o.f, o.ytri, o.ypair)):
                assert np.array_equal(u, v), what
        else:
            for u, v in zip(g, (o.x, o.f, o.ytri, o.ypair)):
                assert _rel(u, v) <= 1e-11, what


def test_full_size_chunglu1000_converged():
    """The benchmark workload solved to convergence on both sides (the
    convergence criteria of Sec. IV-D read as max metric violation <= 1e-4,
    checked every 10 sweeps): the GPU in the launch configuration bench.py
    times (FP64, tile 16, relabeled objects, default sweep form) and the
    oracle's threaded sweep (bit for bit its serial sweep) on the relabeled
    instance.  Same sweep count, LP objective within 1e-6 relative, x within
    1e-7 (rounding of the fused form only, over the whole solve)."""
    import os
    from relabel import deal_labels
    n, d, w, _ = workload("chunglu1000")
    B, tol, every = 16, 1e-4, 10
    lab = deal_labels(n, B)
    iu, ju = np.triu_indices(n, 1)
    a, b = lab[iu], lab[ju]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    pmap = lo * n - lo * (lo + 1) // 2 + (hi - lo - 1)
    dint, wint = np.empty_like(d), np.empty_like(w)
    dint[pmap], wint[pmap] = d, w
    cores = len(os.sched_getaffinity(0))
    o = oracle.State(n, dint, wint, 0.2)
    ko = -1
    for k in range(1, 1001):
        o.sweep_threads(2, B, cores)
        if k % every == 0 and oracle.max_violation(n, o.x, threads=cores) <= tol:
            ko = k
            break
    assert ko > 0
    with _solver(n, d, w, eps=0.2, tile=B, interleave=True, check_every=every) as s:
        conv, kg = s.solve(tol, 1000)
        st = s.check()
        x, _ = s.get_x()
    assert conv and kg == ko and st["max_violation"] <= tol
    oo = o.objectives()
    assert abs(st["lp_objective"] - oo["lp"]) <= 1e-6 * abs(oo["lp"])
    assert abs(st["qp_primal"] - oo["qp_primal"]) <= 1e-6 * abs(oo["qp_primal"])
    assert np.max(np.abs(x - o.x[pmap])) <= 1e-7


def test_full_size_chunglu3000w_two_sweeps_sampled():
    """The precision form's instance (Chung-Lu n = 3000, mean degree 10,
    w ~ U[0.5, 2]) in FP64 on the dense store, in the launch configuration
    bench.py times: two sweeps from the start (the first moves only the pair
    rows, so the second is one sweep from an identical state) against the
    oracle's threaded sweep on the relabeled instance; x and f in full, the
    duals on three sampled ranges of 40000 triplets."""
    import os
    from relabel import deal_labels
    n, d, w, _ = workload("chunglu3000w")
    B = 16
    lab = deal_labels(n, B)
    iu, ju = np.triu_indices(n, 1)
    a, b = lab[iu], lab[ju]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    pmap = lo * n - lo * (lo + 1) // 2 + (hi - lo - 1)
    del iu, ju, a, b, lo, hi
    dint, wint = np.empty_like(d), np.empty_like(w)
    dint[pmap], wint[pmap] = d, w
    cores = len(os.sched_getaffinity(0))
    o = oracle.State(n, dint, wint, 0.2)
    for _ in range(2):
        o.sweep_threads(2, B, cores)
    with _solver(n, d, w, eps=0.2, tile=B, interleave=True) as s:
        s.sweep(2)
        x, f = s.get_x()
        assert _rel(x, o.x[pmap]) <= TOL_SWEEP and _rel(f, o.f[pmap]) <= TOL_SWEEP
        T = n * (n - 1) * (n - 2) // 6
        for first in (0, T // 3, T - 40000):
            yt, _ = s.get_duals(first, 40000, pairs=False)
            ref = np.empty(3 * 40000)
            for q, (i, j, k) in enumerate(_caller_triplets(n, first, 40000)):
                li, lj, lk = lab[i], lab[j], lab[k]
                u, z = min(li, lj, lk), max(li, lj, lk)
                v = li + lj + lk - u - z
                base = 3 * oracle.trank(n, u, v, z)
                for row, out in enumerate((lk, lj, li)):
                    ref[3 * q + row] = o.ytri[base + (0 if out == z else 1 if out == v else 2)]
            assert _rel(yt, ref) <= TOL_SWEEP
        st = s.check()
    assert st["max_violation"] == pytest.approx(oracle.max_violation(n, o.x, threads=cores), abs=1e-12)
