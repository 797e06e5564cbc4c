"""The sparse dual store (store="sparse": per block triple a list of its
nonzero duals, Sec. III-D) against the dense store on the GPU: the same
sweeps in the same order with the same arithmetic, so x, f and all duals
agree bit for bit, whatever the pool capacity (a sweep that overflows the
next pool is undone and run again)."""
import numpy as np
import pytest

from instances import chung_lu, noisy_euclidean, planted_partition, random_dissimilarity

pytestmark = pytest.mark.gpu


def _state(n, d, w, sweeps, **kw):
    import paper_1901_10084_gb300 as cc
    with cc.Solver(n, d, w, **kw) as s:
        s.sweep(sweeps)
        x, f = s.get_x()
        yt, yp = s.get_duals()
        st = s.stats()
        nbytes = s.device_bytes()
    return x, f, yt, yp, st, nbytes


def _equal(a, b):
    for u, v in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(u, v)


CASES = [("cc", 60, 8, False, False), ("cc", 61, 16, True, True), ("cc", 150, 16, False, True),
         ("cc", 97, 32, True, False), ("l2", 70, 16, True, True), ("l2", 90, 8, False, False)]


def _inputs(problem, n, weighted):
    if problem == "l2":
        return random_dissimilarity(n, n, weights=(0.5, 2.0) if weighted else None)
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    return d, w


@pytest.mark.parametrize("variant", [0, 3, 4])
@pytest.mark.parametrize("problem,n,tile,weighted,interleave", CASES)
def test_sparse_store_equals_dense_bitwise(variant, problem, n, tile, weighted, interleave):
    d, w = _inputs(problem, n, weighted)
    kw = dict(tile=tile, interleave=interleave, problem=problem, variant=variant)
    for sweeps in (1, 6):
        dense = _state(n, d, w, sweeps, **kw)
        sparse = _state(n, d, w, sweeps, store="sparse", **kw)
        _equal(sparse, dense)
        assert sparse[4]["dual_nnz"] == int(np.count_nonzero(dense[2]))
        assert dense[4]["dual_nnz"] == -1


@pytest.mark.parametrize("pool", [1, 64, 2000])
def test_pool_overflow_undoes_and_reruns_the_sweep(pool):
    n = 120
    d, w, _ = planted_partition(n, 4, 0.6, 0.15, seed=3)
    dense = _state(n, d, w, 8, tile=16)
    sparse = _state(n, d, w, 8, tile=16, store="sparse", pool_entries=pool)
    _equal(sparse, dense)
    if pool < 2000:
        assert sparse[4]["pool_retries"] > 0


def test_sparse_solve_matches_dense():
    import paper_1901_10084_gb300 as cc
    n, d, w = 200, *chung_lu(200, 2.5, 8.0, seed=5)[:2]
    out = []
    for store in ("dense", "sparse"):
        with cc.Solver(n, d, w, tile=16, store=store, check_every=5) as s:
            conv, k = s.solve(1e-6, 20000)
            st = s.check()
            x, _ = s.get_x()
        out.append((conv, k, st["lp_objective"], x))
    assert out[0][0] and out[1][0] and out[0][1] == out[1][1]
    assert out[0][2] == out[1][2] and np.array_equal(out[0][3], out[1][3])


def test_sparse_dual_ranges():
    import paper_1901_10084_gb300 as cc
    n = 400
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=9)
    T = n * (n - 1) * (n - 2) // 6
    with cc.Solver(n, d, w, tile=16, store="sparse") as s:
        s.sweep(4)
        full, _ = s.get_duals()
        for first, count in ((0, 1000), (T // 3, 5000), (T - 777, 777)):
            part, _ = s.get_duals(first, count, pairs=False)
            np.testing.assert_array_equal(part, full[3 * first: 3 * (first + count)])


def test_sparse_store_memory():
    """n = 800: the dense FP64 store and bitmask take 2.2 GB; the sparse store
    (pools, tables, per-CTA scratch, snapshot) a small fraction of that."""
    import paper_1901_10084_gb300 as cc
    n = 800
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=9)
    with cc.Solver(n, d, w, tile=16, store="sparse") as s, cc.Solver(n, d, w, tile=16) as t:
        s.sweep(10)
        t.sweep(10)
        dense_bytes, sparse_bytes = t.device_bytes(), s.device_bytes()
    assert dense_bytes > 2e9 and sparse_bytes < dense_bytes / 8


def test_unsupported_combinations_are_refused():
    import paper_1901_10084_gb300 as cc
    from paper_1901_10084_gb300 import warmstart
    n = 40
    d, w, _ = planted_partition(n, 2, 0.7, 0.1, seed=1)
    for kw in (dict(exact=True), dict(schedule="summod"),
               dict(schedule="diagonal"), dict(variant=1), dict(variant=2)):
        with pytest.raises(cc.CCError) as e:
            cc.Solver(n, d, w, store="sparse", **kw)
        assert e.value.code == cc.CC_ERR_UNSUPPORTED, kw
    with cc.Solver(n, d, w, store="sparse", tile=8) as s:
        s.sweep(2)
        x, f = s.get_x()
        yt, yp = s.get_duals()
        for call in (lambda: s.set_state(x, f, yt, yp), lambda: s.set_duals(yt, yp),
                     lambda: s.warm_start(warmstart.init_params(0))):
            with pytest.raises(cc.CCError) as e:
                call()
            assert e.value.code == cc.CC_ERR_UNSUPPORTED
    from paper_1901_10084_gb300 import _native
    o = cc.cc_opts_default()
    o.store = _native.CC_STORE_SPARSE
    with pytest.raises(cc.CCError) as e:
        _native.cc_batch_create([n], [d], [w], o)
    assert e.value.code == cc.CC_ERR_UNSUPPORTED


def test_large_instance_beyond_the_dense_store():
    """n = 3000 (the dense FP64 store would need 108 GB): sweeps run, the
    violation falls and the store holds only the nonzero duals."""
    import paper_1901_10084_gb300 as cc
    n = 3000
    d, w = noisy_euclidean(n, 2, 0.2, 4)
    with cc.Solver(n, d, w, problem="l2", tile=16, store="sparse") as s:
        v0 = s.check()["max_violation"]
        s.sweep(3)
        st = s.check()
        nbytes = s.device_bytes()
    assert st["max_violation"] < v0
    assert 0 < st["dual_nnz"] < 3 * n * (n - 1) * (n - 2) // 6 // 100
    assert nbytes < 8e9


@pytest.mark.parametrize("n,tile,weighted,interleave", [(61, 16, True, True), (150, 8, False, False),
                                                      (97, 32, True, False)])
def test_sparse_store_in_the_fp32_bulk_form(n, tile, weighted, interleave):
    """FP32 bulk sweeps, the FP64 switch (the resync reads the sparse lists in
    the dense resync's order) and FP64 sweeps after it: the same values as
    the dense store, bit for bit; the refined solve too."""
    import paper_1901_10084_gb300 as cc
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n + 2, weights=(0.5, 2.0) if weighted else None)
    kw = dict(tile=tile, interleave=interleave, precision="fp32_refine")
    out = []
    for store in ("dense", "sparse"):
        with cc.Solver(n, d, w, store=store, pool_entries=128, **kw) as s:
            s.sweep(6)
            a = (*s.get_x(), *s.get_duals())
            s.refine_fp64()
            b = (*s.get_x(), *s.get_duals())
            s.sweep(3)
            c = (*s.get_x(), *s.get_duals())
        with cc.Solver(n, d, w, store=store, check_every=5, **kw) as s:
            conv, k = s.solve(1e-6, 20000)
            st = s.stats()
            sol = (conv, k, st["fp32_sweeps"], s.get_x()[0])
        out.append((a, b, c, sol))
    for u, v in zip(out[0][:3], out[1][:3]):
        for p, q in zip(u, v):
            np.testing.assert_array_equal(p, q)
    assert out[0][3][:3] == out[1][3][:3] and out[0][3][0]
    np.testing.assert_array_equal(out[0][3][3], out[1][3][3])


# ------------------------------------------------------------- against the oracle

SPARSE_ORACLE_CASES = [(61, 8, False, 5), (61, 16, True, 12), (61, 32, True, 20), (97, 16, True, 20),
                       (150, 32, False, 8)]


@pytest.mark.parametrize("n,tile,weighted,sweeps", SPARSE_ORACLE_CASES)
def test_sparse_store_matches_the_oracle_over_many_sweeps(n, tile, weighted, sweeps):
    """The sparse store's own staging, gather and pool code against the
    oracle (schedule 2 on consecutive blocks, the order the handle walks with
    interleave off): after `sweeps` sweeps from the start, x, f, every
    triangle dual (canonical order) and every pair dual element by element.
    The fused row form differs from the oracle's row only in rounding, so the
    states agree to rounding level (1e-11 in ||.||_inf / max(||.||_inf, 1)
    after up to 20 sweeps, as for the dense store); the support of the duals
    (which duals are nonzero) is compared exactly where the oracle's duals
    are away from zero."""
    import oracle
    import paper_1901_10084_gb300 as cc
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n + tile, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    for _ in range(sweeps):
        o.sweep(2, tile)
    with cc.Solver(n, d, w, eps=0.2, tile=tile, store="sparse", interleave=False, pool_entries=256) as s:
        s.sweep(sweeps)
        x, f = s.get_x()
        yt, yp = s.get_duals()
        st = s.stats()
    rel = lambda a, b: float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0))
    assert rel(x, o.x) <= 1e-11 and rel(f, o.f) <= 1e-11
    assert rel(yt, o.ytri) <= 1e-11 and rel(yp, o.ypair) <= 1e-11
    away = np.abs(o.ytri) > 1e-9
    assert np.array_equal(yt[away] != 0, np.ones(int(away.sum()), dtype=bool))
    assert st["dual_nnz"] == int(np.count_nonzero(yt))
    assert np.count_nonzero(o.ytri) > 0


def test_sparse_store_late_solve_matches_the_oracle():
    """Late in the solve, where most nonzero duals sit and the row-skip
    filters decide differently than early on: 60 sweeps of the sparse store
    and of the oracle from the start (n = 200, weighted, tile 16), then the
    state element by element."""
    import oracle
    import paper_1901_10084_gb300 as cc
    n = 200
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=77, weights=(0.5, 2.0))
    o = oracle.State(n, d, w, 0.2)
    for _ in range(60):
        o.sweep(2, 16)
    with cc.Solver(n, d, w, eps=0.2, tile=16, store="sparse", interleave=False) as s:
        s.sweep(60)
        x, f = s.get_x()
        yt, yp = s.get_duals()
    rel = lambda a, b: float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0))
    assert rel(x, o.x) <= 1e-10 and rel(f, o.f) <= 1e-10
    assert rel(yt, o.ytri) <= 1e-10 and rel(yp, o.ypair) <= 1e-10
    assert np.count_nonzero(o.ytri) > 1000
