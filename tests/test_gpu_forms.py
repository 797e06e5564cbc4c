"""The FP64 sweep's per-warp form (default) and compacted form (variant 1)
update the same triplets with the same arithmetic, so their iterates, duals
and nonzero-dual masks agree bit for bit; and a sweep is deterministic (the
dataflow order inside a sub-phase never changes a result).  GPU."""
import numpy as np
import pytest

from instances import chung_lu, planted_partition

pytestmark = pytest.mark.gpu


def _run(n, d, w, sweeps, solve=None, **kw):
    import paper_1901_10084_gb300 as cc
    with cc.Solver(n, d, w, **kw) as s:
        if solve is None:
            s.sweep(sweeps)
        else:
            s.solve(solve, sweeps)
        x, f = s.get_x()
        yt, yp = s.get_duals()
        st = s.stats()
    return x, f, yt, yp, st


CASES = [(60, 8, False, False), (61, 16, False, True), (130, 16, True, False), (200, 16, False, True),
         (97, 32, True, True), (300, 32, False, False)]


@pytest.mark.parametrize("n,tile,weighted,interleave", CASES)
def test_per_warp_and_compacted_fp64_forms_agree_bitwise(n, tile, weighted, interleave):
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n + tile, weights=(0.5, 2.0) if weighted else None)
    kw = dict(tile=tile, interleave=interleave)
    a = _run(n, d, w, 25, variant=0, **kw)
    b = _run(n, d, w, 25, variant=1, **kw)
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("n,tile,weighted,interleave", CASES[1:4])
def test_sweeps_are_deterministic(n, tile, weighted, interleave, precision):
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n + 1, weights=(0.5, 2.0) if weighted else None)
    kw = dict(tile=tile, interleave=interleave, precision=precision)
    a = _run(n, d, w, 30, **kw)
    b = _run(n, d, w, 30, **kw)
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)


def test_fp32_refine_solve_is_deterministic_and_forms_agree():
    n = 250
    d, w, _ = planted_partition(n, 5, 0.6, 0.1, seed=8)
    runs = [_run(n, d, w, 2000, solve=1e-6, tile=16, precision="fp32_refine", variant=v) for v in (0, 0, 1)]
    for r in runs[1:]:
        for u, v in zip(runs[0][:4], r[:4]):
            assert np.array_equal(u, v)
        assert r[4]["sweeps"] == runs[0][4]["sweeps"] and r[4]["fp32_sweeps"] == runs[0][4]["fp32_sweeps"]


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("n,tile,weighted,interleave", CASES)
def test_filtered_forms_equal_the_unfiltered_sweep(n, tile, weighted, interleave, precision):
    """Variant 4 updates every triplet and every row; the float filters only
    skip updates that are no-ops, so the filtered sweeps give the same values
    (x + 0 may turn -0.0 into +0.0, which compares equal)."""
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=3 * n + tile, weights=(0.5, 2.0) if weighted else None)
    kw = dict(tile=tile, interleave=interleave, precision=precision)
    ref = _run(n, d, w, 20, variant=4, **kw)
    for v in (0, 1, 3):
        got = _run(n, d, w, 20, variant=v, **kw)
        for u, r in zip(got[:4], ref[:4]):
            assert np.array_equal(u, r), v
    if tile <= 16:
        got = _run(n, d, w, 20, variant=2, **kw)
        for u, r in zip(got[:4], ref[:4]):
            assert np.array_equal(u, r)


@pytest.mark.parametrize("store", ["dense", "sparse"])
@pytest.mark.parametrize("n,tile,weighted", [(60, 8, False), (130, 16, True), (97, 32, False)])
def test_first_sweep_shortcut_is_exact(store, n, tile, weighted):
    """From Algorithm 1's start every metric row is a no-op, so the first
    sweep runs only the pair rows; it must equal a full first sweep (forced
    by setting the same start state, which turns the shortcut off) bit for
    bit, and the oracle's first sweep to 1e-12 (the fused rounding)."""
    import oracle
    import paper_1901_10084_gb300 as cc
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    P = len(d)
    T = n * (n - 1) * (n - 2) // 6
    o = oracle.State(n, d, w, 0.2)
    x0, f0 = o.x.copy(), o.f.copy()
    o.sweep(2, tile)
    kw = dict(tile=tile, interleave=False)
    a = _run(n, d, w, 1, **kw)
    with cc.Solver(n, d, w, **kw) as s:
        s.set_state(x0, f0, np.zeros(3 * T), np.zeros(2 * P))
        s.sweep(1)
        x, f = s.get_x()
        yt, yp = s.get_duals()
    for u, v in zip(a[:4], (x, f, yt, yp)):
        assert np.array_equal(u, v)
    assert np.max(np.abs(a[0] - o.x)) <= 1e-12 and np.max(np.abs(a[1] - o.f)) <= 1e-12
    if store == "sparse":
        b = _run(n, d, w, 3, store="sparse", **kw)
        c = _run(n, d, w, 3, **kw)
        for u, v in zip(b[:4], c[:4]):
            assert np.array_equal(u, v)


def test_random_configurations_equal_the_unfiltered_sweep():
    """Seeded fuzzing of the exactness claim: random sizes (including tiny and
    ragged ones), tiles, weights, relabeling, problems, stores and precision
    forms; the default sweep must equal the unfiltered one bit for bit."""
    from instances import random_dissimilarity
    rng = np.random.default_rng(2024)
    for case in range(24):
        problem = "l2" if rng.random() < 0.3 else "cc"
        n = int(rng.choice([3, 4, 5, 17, 33, 64, 65, 97, 130, 211]))
        tile = int(rng.choice([8, 16, 32]))
        weighted = bool(rng.random() < 0.5)
        store = "sparse" if rng.random() < 0.4 else "dense"
        precision = "fp32_refine" if (problem == "cc" and rng.random() < 0.3) else "fp64"
        interleave = bool(rng.random() < 0.5)
        sweeps = int(rng.integers(1, 12))
        seed = int(rng.integers(0, 10**6))
        if problem == "l2":
            d, w = random_dissimilarity(n, seed, weights=(0.5, 2.0) if weighted else None)
        else:
            d, w, _ = chung_lu(n, 2.5, 8.0, seed=seed, weights=(0.5, 2.0) if weighted else None)
        kw = dict(tile=tile, interleave=interleave, problem=problem, precision=precision, store=store)
        a = _run(n, d, w, sweeps, variant=0, **kw)
        b = _run(n, d, w, sweeps, variant=4, **kw)
        for u, v in zip(a[:4], b[:4]):
            assert np.array_equal(u, v), (case, kw, n, sweeps)


def test_automatic_sweep_form_gives_the_same_values():
    """opts.variant = -1 (the default) picks form 0 or 3 per instance and
    precision; the forms give the same values, so the automatic choice equals
    form 0 bit for bit.  A small instance (one phase holds few block triples)
    keeps form 0."""
    import numpy as np
    import paper_1901_10084_gb300 as cc
    from instances import chung_lu
    d, w, _ = chung_lu(90, 2.5, 8.0, seed=3)
    with cc.Solver(90, d, w, tile=16) as s:
        s.sweep(2)
        assert s.stats()["variant"] == 0
    n = 2000
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=4)
    for prec in ("fp64", "fp32_refine"):
        out = []
        for v in (-1, 0):
            with cc.Solver(n, d, w, tile=16, precision=prec, variant=v) as s:
                s.sweep(4)
                st = s.stats()
                out.append((s.get_x()[0], st["variant"]))
        assert out[0][1] in (0, 3) and out[1][1] == 0
        assert np.array_equal(out[0][0], out[1][0])
