"""Traced dataflow sweeps on the GPU: no block triple's dependencies are met
before every predecessor (the previous phase's visitor of each of its tiles)
has finished processing, and the longest chain spans every phase."""
import pytest

from instances import chung_lu, planted_partition

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,tile,precision", [(300, 16, "fp64"), (170, 8, "fp64"), (300, 16, "fp32_refine"),
                                             (400, 32, "fp64")])
def test_traced_sweeps_respect_the_dataflow(n, tile, precision):
    import paper_1901_10084_gb300 as cc
    from paper_1901_10084_gb300 import chain
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n)
    with cc.Solver(n, d, w, tile=tile, precision=precision, trace=True) as s:
        for _ in range(3):
            s.sweep(4)
            r = chain.critical_path(s.trace(), n, tile)
            assert r["started_early"] == 0
            assert r["chain_items"] == -(-n // tile)
            assert 0 < r["chain_frac"] <= 1 and r["span_us"] > 0


def test_sparse_store_trace_respects_the_dataflow():
    import paper_1901_10084_gb300 as cc
    from paper_1901_10084_gb300 import chain
    n = 260
    d, w, _ = planted_partition(n, 5, 0.6, 0.1, seed=2)
    with cc.Solver(n, d, w, tile=16, store="sparse", trace=True) as s:
        s.sweep(6)
        assert chain.critical_path(s.trace(), n, 16)["started_early"] == 0
