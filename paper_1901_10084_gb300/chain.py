"""Dependency-chain analysis of one traced dataflow sweep (host only).

A sweep of the tiled schedule (Sec. III-C, the b x b tiling) is a dataflow:
block triple (I, J, K) of phase g = (I + J + K) mod Nb may run once each of
its tiles (I, J), (I, K), (J, K) has been visited by phase g - 1, and the
pair item of a tile once the tile has all Nb visits.  However many CTAs run,
a sweep cannot end before its longest chain of dependent items has run one
after the other.  With the per-item timestamps of ``Solver.trace()`` this
module rebuilds the work list in the library's order, finds that chain and
splits the sweep's span into the chain's own work and the hand-offs between
its items.  Nothing here touches the GPU.
"""
from __future__ import annotations

import numpy as np


def _bsize(n: int, B: int, I: int) -> int:
    return min(B, n - I * B)


def _count(n: int, B: int, I: int, J: int, K: int) -> int:
    def c2(m):
        return m * (m - 1) // 2 if m >= 2 else 0

    def c3(m):
        return m * (m - 1) * (m - 2) // 6 if m >= 3 else 0
    if I == J == K:
        return c3(_bsize(n, B, I))
    if I == J:
        return c2(_bsize(n, B, I)) * _bsize(n, B, K)
    if J == K:
        return _bsize(n, B, I) * c2(_bsize(n, B, J))
    return _bsize(n, B, I) * _bsize(n, B, J) * _bsize(n, B, K)


def work_list(n: int, B: int):
    """(block triples, phases, tiles): the sweep's work items in the order the
    library hands them out -- phase by phase, inside a phase the block triples
    with more triplets first (ties in (I, J) order) -- then one pair item per
    tile (I <= J, row-major)."""
    nb = -(-n // B)
    items, phase = [], []
    for g in range(nb):
        ph = []
        for I in range(nb):
            for J in range(I, nb):
                K = (g - I - J) % nb
                if K >= J:
                    ph.append((-_count(n, B, I, J, K), I, J, K))
        ph.sort(key=lambda e: e[0])          # stable: (I, J) order among equals
        for _, I, J, K in ph:
            items.append((I, J, K))
            phase.append(g)
    tiles = [(I, J) for I in range(nb) for J in range(I, nb)]
    return items, phase, tiles


def dependencies(n: int, B: int):
    """For every work item (block triples, then pair items), the items it
    waits for: the previous phase's visitor of each of its tiles."""
    items, phase, tiles = work_list(n, B)
    nb = -(-n // B)
    visitor, deps = {}, []
    for w, ((I, J, K), g) in enumerate(zip(items, phase)):
        ts = sorted({(I, J), (I, K), (J, K)})
        deps.append([visitor[(g - 1, t)] for t in ts] if g > 0 else [])
        for t in ts:
            visitor[(g, t)] = w
    for t in tiles:
        deps.append([visitor[(nb - 1, t)]])
    return deps, len(items)


def critical_path(trace: np.ndarray, n: int, B: int) -> dict:
    """Longest chain of a traced sweep.  ``trace``: the (items, 6) array of
    ``Solver.trace()`` (taken, dependencies met, processed, released in ns;
    counts; CTA).  A block triple's work is its release minus the moment its
    dependencies were met; pair items carry only the taken timestamp and
    count with no work (they end the sweep, one short step per tile).
    Returns the span (first item taken to last release), the chain (item
    indices), its work, the rest of the span (hand-offs between the chain's
    items), and the number of block triples whose dependencies were met
    before a predecessor had finished processing (0 for a valid dataflow)."""
    tr = np.asarray(trace, dtype=np.int64)
    deps, nbt = dependencies(n, B)
    if tr.shape[0] != len(deps):
        raise ValueError(f"trace has {tr.shape[0]} items, the schedule {len(deps)}")
    t0 = tr[:nbt, 0].min()
    t = tr[:, :4] - t0
    end = np.zeros(len(deps))
    end[:nbt] = t[:nbt, 3]
    end[nbt:] = t[nbt:, 0]
    work = np.zeros(len(deps))
    work[:nbt] = np.maximum(t[:nbt, 3] - t[:nbt, 1], 0)
    fin = np.zeros(len(deps))
    early = 0
    for w in range(len(deps)):
        if w < nbt and any(t[w, 1] < t[p, 2] for p in deps[w]):
            early += 1
        fin[w] = max((fin[p] for p in deps[w]), default=0.0) + work[w]
    w = int(np.argmax(fin[:nbt]))
    chain = [w]
    while deps[w]:
        w = max(deps[w], key=lambda p: fin[p])
        chain.append(w)
    chain.reverse()
    span = float(end[:nbt].max())
    chain_work = float(work[chain].sum())
    return {"span_us": span / 1e3, "chain_items": len(chain), "chain_work_us": chain_work / 1e3,
            "handoff_us": (span - chain_work) / 1e3, "chain_frac": chain_work / span if span > 0 else 0.0,
            "item_work_mean_us": float(work[:nbt].mean()) / 1e3,
            "chain_item_work_mean_us": float(work[chain].mean()) / 1e3,
            "started_early": early, "chain": chain}


def simulate(trace: np.ndarray, n: int, B: int, slots=None, hop_ns: float = 1000.0) -> float:
    """Span (us) of a model sweep with the traced work of each item: `slots`
    CTAs (None: one per item) take the items in list order, an item starts
    when it is taken and `hop_ns` after its last predecessor's release, and
    holds its CTA for its work.  With unlimited slots this is the longest
    chain with a fixed hand-off per hop."""
    import heapq
    tr = np.asarray(trace, dtype=np.int64)
    deps, nbt = dependencies(n, B)
    if tr.shape[0] != len(deps):
        raise ValueError(f"trace has {tr.shape[0]} items, the schedule {len(deps)}")
    work = np.zeros(len(deps))
    work[:nbt] = np.maximum(tr[:nbt, 3] - tr[:nbt, 1], 0)
    free = [0.0] * (len(deps) if slots is None else int(slots))
    heapq.heapify(free)
    rel = np.zeros(len(deps))
    for w in range(len(deps)):
        taken = heapq.heappop(free)
        start = max([taken] + [rel[p] + hop_ns for p in deps[w]])
        rel[w] = start + work[w]
        heapq.heappush(free, rel[w])
    return float(rel.max()) / 1e3
