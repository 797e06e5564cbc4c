"""Pair-only passes (cc_pair_passes: Algorithm 1's row step on the pair rows
alone, Hildreth's coordinate ascent on the pair block of the dual, Sec. II-B)
against the oracle's single-pair visits repeated pass by pass: the exact form
bit for bit, the fused form within 1e-12 relative, FP32 state within FP32
rounding; the sparse store as the dense one; l2 nearness untouched."""
import numpy as np
import pytest

import oracle
from instances import chung_lu, random_dissimilarity

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0)) if a.size else 0.0


def _oracle_state(n, d, w, sweeps, tile):
    o = oracle.State(n, d, w, 0.2)
    for _ in range(sweeps):
        o.sweep(2, tile)
    return o


def _oracle_passes(o, passes):
    for _ in range(passes):
        for p in range(len(o.x)):
            o.visit_pair(p)


@pytest.mark.parametrize("exact,n,tile,weighted,passes", [
    (True, 40, 8, False, 1), (True, 61, 16, True, 5), (True, 97, 16, True, 16),
    (False, 40, 8, False, 1), (False, 61, 16, True, 5), (False, 97, 32, True, 16)])
def test_pair_passes_match_the_oracle(exact, n, tile, weighted, passes):
    import paper_1901_10084_gb300 as cc
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = _oracle_state(n, d, w, 3, tile)
    with cc.Solver(n, d, w, eps=0.2, tile=tile, exact=exact, interleave=False) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        yt0, _ = s.get_duals()
        s.pair_passes(passes)
        _oracle_passes(o, passes)
        x, f = s.get_x()
        yt, yp = s.get_duals()
        assert s.stats()["sweeps"] == 0
    np.testing.assert_array_equal(yt, yt0)   # triangle duals untouched
    if exact:
        np.testing.assert_array_equal(yt, o.ytri)
        np.testing.assert_array_equal(x, o.x)
        np.testing.assert_array_equal(f, o.f)
        np.testing.assert_array_equal(yp, o.ypair)
    else:
        assert _rel(x, o.x) <= 1e-12 and _rel(f, o.f) <= 1e-12 and _rel(yp, o.ypair) <= 1e-12


def test_pair_passes_then_sweeps_track_the_oracle():
    """From the initial state (where the first-sweep shortcut would apply) the
    passes leave x != 0, and the following sweeps are the oracle's."""
    import paper_1901_10084_gb300 as cc
    n = 70
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=3)
    o = oracle.State(n, d, w, 0.2)
    with cc.Solver(n, d, w, eps=0.2, tile=16, exact=True, interleave=False) as s:
        s.pair_passes(4)
        _oracle_passes(o, 4)
        s.sweep(2)
        for _ in range(2):
            o.sweep(2, 16)
        x, f = s.get_x()
        yt, yp = s.get_duals()
    np.testing.assert_array_equal(x, o.x)
    np.testing.assert_array_equal(f, o.f)
    np.testing.assert_array_equal(yt, o.ytri)
    np.testing.assert_array_equal(yp, o.ypair)


def test_pair_passes_in_fp32_state():
    import paper_1901_10084_gb300 as cc
    n = 80
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=8, weights=(0.5, 2.0))
    with cc.Solver(n, d, w, eps=0.2, tile=16, precision="fp32_refine", interleave=False) as s:
        s.sweep(3)
        x0, f0 = s.get_x()
        yt, yp = s.get_duals()
        o = oracle.State(n, d, w, 0.2)
        o.x[:], o.f[:], o.ytri[:], o.ypair[:] = x0, f0, yt, yp
        s.pair_passes(6)
        _oracle_passes(o, 6)
        x, f = s.get_x()
        _, yp1 = s.get_duals()
    assert _rel(x, o.x) <= 1e-5 and _rel(f, o.f) <= 1e-5 and _rel(yp1, o.ypair) <= 1e-5


def test_sparse_store_equals_dense():
    import paper_1901_10084_gb300 as cc
    n = 90
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=4)
    out = []
    for store in ("dense", "sparse"):
        with cc.Solver(n, d, w, tile=16, store=store) as s:
            s.sweep(3)
            s.pair_passes(7)
            s.sweep(2)
            out.append((*s.get_x(), *s.get_duals()))
    for u, v in zip(*out):
        np.testing.assert_array_equal(u, v)


def test_l2_has_no_pair_rows_and_other_schedules_are_refused():
    import paper_1901_10084_gb300 as cc
    n = 40
    d, w = random_dissimilarity(n, 2)
    with cc.Solver(n, d, w, problem="l2", tile=8) as s:
        s.sweep(2)
        x0, _ = s.get_x()
        s.pair_passes(5)
        x1, _ = s.get_x()
    np.testing.assert_array_equal(x0, x1)
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=1)
    with cc.Solver(n, d, w, schedule="summod") as s:
        with pytest.raises(cc.CCError) as e:
            s.pair_passes(1)
        assert e.value.code == cc.CC_ERR_UNSUPPORTED
        with pytest.raises(cc.CCError) as e:
            s.pair_passes(-1)
        assert e.value.code == cc.CC_ERR_ARG
