"""Host-side dependency-chain analysis of a traced sweep
(paper_1901_10084_gb300.chain): the work list against a brute-force
enumeration of the tiled schedule (Sec. III-C), the dependencies against the
tile visits, and the longest chain of synthetic traces against networkx."""
import itertools

import networkx as nx
import numpy as np
import pytest

from paper_1901_10084_gb300 import chain


@pytest.mark.parametrize("n,B", [(3, 8), (17, 8), (40, 8), (50, 16), (33, 16), (70, 32)])
def test_work_list_is_the_tiled_schedule(n, B):
    nb = -(-n // B)
    items, phase, tiles = chain.work_list(n, B)
    want = sorted((I, J, K) for I, J, K in itertools.combinations_with_replacement(range(nb), 3))
    assert sorted(items) == want
    assert all((I + J + K) % nb == g for (I, J, K), g in zip(items, phase))
    assert phase == sorted(phase)
    size = lambda I: min(B, n - I * B)
    cnt = [len([t for t in itertools.product(range(size(I)), range(size(J)), range(size(K)))
                if I * B + t[0] < J * B + t[1] < K * B + t[2]]) for I, J, K in items]
    for g in range(nb):
        c = [x for x, p in zip(cnt, phase) if p == g]
        assert c == sorted(c, reverse=True)
    assert tiles == [(I, J) for I in range(nb) for J in range(I, nb)]


@pytest.mark.parametrize("n,B", [(40, 8), (50, 16)])
def test_dependencies_are_the_previous_visits(n, B):
    nb = -(-n // B)
    items, phase, tiles = chain.work_list(n, B)
    deps, nbt = chain.dependencies(n, B)
    assert nbt == len(items) and len(deps) == nbt + len(tiles)
    for g in range(nb):   # every tile visited exactly once per phase
        seen = [t for (I, J, K), p in zip(items, phase) if p == g for t in {(I, J), (I, K), (J, K)}]
        assert sorted(seen) == tiles
    for w, (I, J, K) in enumerate(items):
        mine = {(I, J), (I, K), (J, K)}
        assert len(deps[w]) == (len(mine) if phase[w] > 0 else 0)
        for p in deps[w]:
            a, b, c = items[p]
            assert phase[p] == phase[w] - 1 and mine & {(a, b), (a, c), (b, c)}
    for tl, t in enumerate(tiles):
        (p,) = deps[nbt + tl]
        a, b, c = items[p]
        assert phase[p] == nb - 1 and t in {(a, b), (a, c), (b, c)}


def _synthetic_trace(n, B, seed, hop=300):
    """Timestamps of a dataflow with unlimited CTAs: an item's dependencies
    are met `hop` ns after its last predecessor's release."""
    rng = np.random.default_rng(seed)
    deps, nbt = chain.dependencies(n, B)
    work = rng.integers(1000, 20000, nbt)
    tr = np.zeros((len(deps), 6), dtype=np.int64)
    base = 10_000
    for w in range(len(deps)):
        ready = max((tr[p, 3] for p in deps[w]), default=base) + (hop if deps[w] else 0)
        tr[w, 0] = ready - 50
        if w < nbt:
            tr[w, 1] = ready
            tr[w, 2] = ready + work[w] - 100
            tr[w, 3] = ready + work[w]
    return tr, work, deps, nbt


@pytest.mark.parametrize("n,B,seed", [(40, 8, 1), (50, 16, 2), (90, 16, 3)])
def test_longest_chain_matches_networkx(n, B, seed):
    tr, work, deps, nbt = _synthetic_trace(n, B, seed)
    g = nx.DiGraph()
    for w in range(nbt):
        g.add_node(w)
        for p in deps[w]:
            g.add_edge(p, w, weight=int(work[w]))
    for w in range(nbt):   # a source edge carrying each item's own work
        g.add_edge("s", w, weight=int(work[w]))
    best = nx.dag_longest_path_length(g, weight="weight")
    r = chain.critical_path(tr, n, B)
    assert r["chain_work_us"] * 1e3 == pytest.approx(best)
    assert r["started_early"] == 0
    assert r["chain_items"] == -(-n // B)          # one block triple per phase
    assert 0 < r["chain_frac"] <= 1
    assert r["handoff_us"] == pytest.approx(r["span_us"] - r["chain_work_us"])


def test_an_item_started_before_its_predecessor_is_reported():
    n, B = 40, 8
    tr, work, deps, nbt = _synthetic_trace(n, B, 4)
    w = next(i for i in range(nbt) if deps[i])
    p = deps[w][0]
    tr[w, 1] = tr[p, 2] - 1
    assert chain.critical_path(tr, n, B)["started_early"] == 1


def test_trace_of_another_size_is_refused():
    tr, *_ = _synthetic_trace(40, 8, 5)
    with pytest.raises(ValueError):
        chain.critical_path(tr, 41, 8)


@pytest.mark.parametrize("n,B,hop", [(40, 8, 0.0), (50, 16, 700.0)])
def test_model_with_unlimited_slots_is_the_longest_chain(n, B, hop):
    tr, work, deps, nbt = _synthetic_trace(n, B, 6)
    g = nx.DiGraph()
    for w in range(len(deps)):
        ww = int(work[w]) if w < nbt else 0
        g.add_edge("s", w, weight=ww)
        for p in deps[w]:
            g.add_edge(p, w, weight=ww + hop)
    best = nx.dag_longest_path_length(g, weight="weight")
    assert chain.simulate(tr, n, B, None, hop) * 1e3 == pytest.approx(best)


def test_model_with_one_slot_runs_the_items_one_after_another():
    n, B, hop = 40, 8, 500.0
    tr, work, deps, nbt = _synthetic_trace(n, B, 7)
    t, rel = 0.0, {}
    for w in range(len(deps)):
        t = max([t] + [rel[p] + hop for p in deps[w]]) + (work[w] if w < nbt else 0)
        rel[w] = t
    assert chain.simulate(tr, n, B, 1, hop) * 1e3 == pytest.approx(t)
    assert chain.simulate(tr, n, B, 1, hop) >= chain.simulate(tr, n, B, 4, hop) >= chain.simulate(tr, n, B, None, hop)
