"""Pins for the oracle's schedules (Sec. III-A/B/C): every triplet exactly
once per sweep, the phase counts the paper states, and conflict-freeness of
the units that may run at the same time."""
import itertools
import json
import os
from collections import defaultdict

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pairs(t):
    _, i, j, k = t
    return ((i, j), (i, k), (j, k))


@pytest.mark.parametrize("n", list(range(3, 31)) + [37, 48, 61])
@pytest.mark.parametrize("schedule,tile", [(0, 0), (1, 0), (2, 2), (2, 3), (2, 5), (2, 8)])
def test_each_triplet_exactly_once(n, schedule, tile):
    rec = oracle.order(n, schedule, tile)
    got = sorted(tuple(r[1:]) for r in rec.tolist())
    assert got == list(itertools.combinations(range(n), 3))


@pytest.mark.parametrize("n", range(3, 40))
def test_phase_counts(n):
    assert oracle.num_phases(n, 0) == 2 * n - 5       # diagonals n+1..4, then n+2..2n-2
    assert oracle.num_phases(n, 1) == n
    for B in (2, 4, 7):
        assert oracle.num_phases(n, 2, B) == -(-n // B)


@pytest.mark.parametrize("n", [3, 4, 9, 12, 13, 20, 33])
def test_schedule0_phases_are_the_diagonals(n):
    """Phases of schedule 0 are the diagonals i+k = const (1-based): first
    n+1 down to 4, then n+2 up to 2n-2; inside a phase the sets S_{i,k} come
    in ascending i, and a set's triplets in ascending j."""
    rec = oracle.order(n, 0).tolist()
    sig = [n + 1 - t for t in range(n - 2)] + [n + 2 + t for t in range(n - 3)]
    by_phase = defaultdict(list)
    for ph, i, j, k in rec:
        by_phase[ph].append((i, j, k))
    assert sorted(by_phase) == list(range(len(sig)))
    for ph, trip in by_phase.items():
        assert all((i + 1) + (k + 1) == sig[ph] for i, j, k in trip)
        keys = [(i, j) for i, j, k in trip]
        assert keys == sorted(keys)


def test_paper_counts_n12():
    g = json.load(open(os.path.join(GOLD, "schedule_counts.json")))
    n = g["n"]
    rec = oracle.order(n, 0).tolist()
    nph = oracle.num_phases(n, 0)
    assert nph == g["first_loop_diagonals"] + g["second_loop_diagonals"]
    main = [r for r in rec if r[0] == 0]
    sets = defaultdict(int)
    order = []
    for _, i, j, k in main:
        key = (i + 1, k + 1)
        if key not in sets:
            order.append(key)
        sets[key] += 1
    assert [list(s) for s in order] == g["main_diagonal_sets"]
    assert [sets[s] for s in order] == g["main_diagonal_set_sizes"]


@pytest.mark.parametrize("n", [3, 5, 8, 12, 17, 24, 31])
def test_schedule0_sets_on_a_diagonal_are_disjoint(n):
    """Different sets S_{i,k} of one diagonal share at most one index, hence
    no pair; inside a set every triplet shares the pair (i,k) only."""
    rec = oracle.order(n, 0).tolist()
    owner = {}
    for t in rec:
        ph, i, j, k = t
        for pq in _pairs(t):
            key = (ph, pq)
            if key in owner:
                assert owner[key] == (i, k) and pq == (i, k)
            owner[key] = (i, k)


@pytest.mark.parametrize("n", list(range(3, 26)) + [30, 36, 45])
def test_schedule1_phase_touches_each_pair_once(n):
    rec = oracle.order(n, 1).tolist()
    seen = set()
    for t in rec:
        for pq in _pairs(t):
            key = (t[0], pq)
            assert key not in seen
            seen.add(key)
        assert (t[1] + t[2] + t[3]) % n == t[0]


@pytest.mark.parametrize("n,B", [(3, 2), (9, 2), (10, 3), (16, 4), (23, 4), (29, 5), (40, 8), (33, 16)])
def test_schedule2_blocks_and_subphases_are_conflict_free(n, B):
    """Block triples of one phase touch disjoint pairs; inside a block triple
    the triplets of one sub-phase touch disjoint pairs."""
    rec = oracle.order(n, 2, B).tolist()
    pair_owner = {}
    sub_seen = set()
    for t in rec:
        ph, i, j, k = t
        bt = (i // B, j // B, k // B)
        assert sum(bt) % (-(-n // B)) == ph
        sub = (i % B + j % B + k % B) % B
        for pq in _pairs(t):
            key = (ph, pq)
            if key in pair_owner:
                assert pair_owner[key] == bt
            pair_owner[key] = bt
            skey = (bt, sub, pq)
            assert skey not in sub_seen
            sub_seen.add(skey)


@pytest.mark.parametrize("n,B", [(20, 4), (33, 8)])
def test_schedule2_subphases_in_order(n, B):
    """Inside a block triple the sub-phase index never decreases."""
    rec = oracle.order(n, 2, B).tolist()
    last = {}
    for ph, i, j, k in rec:
        bt = (i // B, j // B, k // B)
        sub = (i % B + j % B + k % B) % B
        assert sub >= last.get(bt, -1)
        last[bt] = sub


def _ranks(n, rec):
    """Lexicographic rank of each (i, j, k) row of an order record (vectorized)."""
    i, j, k = (rec[:, c].astype(np.int64) for c in (1, 2, 3))
    c3 = lambda m: m * (m - 1) * (m - 2) // 6
    c2 = lambda m: m * (m - 1) // 2
    return (c3(n) - c3(n - i)) + (c2(n - 1 - i) - c2(n - j)) + (k - j - 1)


@pytest.mark.parametrize("n", [99, 150, 200])
@pytest.mark.parametrize("schedule,tile", [(0, 0), (1, 0), (2, 16)])
def test_large_n_every_triplet_once_and_phases_conflict_free(n, schedule, tile):
    """Sizes up to n = 200 (n = 99 and 150 are multiples of 3): every i<j<k
    exactly once (the canonical ranks are a permutation, checked against
    oracle.trank on a sample), and inside a phase no pair is touched twice,
    except within one set S_{i,k} of schedule 0, whose triplets share x_ik
    and run in order."""
    rec = oracle.order(n, schedule, tile).astype(np.int64)
    T = n * (n - 1) * (n - 2) // 6
    assert rec.shape[0] == T
    assert np.all((rec[:, 1] < rec[:, 2]) & (rec[:, 2] < rec[:, 3]))
    r = _ranks(n, rec)
    assert np.array_equal(np.sort(r), np.arange(T))
    for t in np.random.default_rng(n).integers(0, T, 20):
        assert oracle.trank(n, *(int(v) for v in rec[t, 1:])) == r[t]
    ph, i, j, k = rec[:, 0], rec[:, 1], rec[:, 2], rec[:, 3]
    pid = lambda a, b: a * n + b
    if schedule == 0:   # pairs (i, j) and (j, k) once per phase; (i, k) once per set
        keys = np.concatenate([ph * n * n + pid(i, j), ph * n * n + pid(j, k)])
        assert np.unique(keys).size == keys.size
        setkey = ph * n * n + pid(i, k)
        starts = np.r_[True, setkey[1:] != setkey[:-1]]
        assert np.unique(setkey[starts]).size == starts.sum()     # each set contiguous, once
    elif schedule == 1:
        keys = np.concatenate([ph * n * n + pid(i, j), ph * n * n + pid(i, k), ph * n * n + pid(j, k)])
        assert np.unique(keys).size == keys.size
        assert np.all((i + j + k) % n == ph)
    else:               # tiled: phase x sub-phase units touch each pair once
        B = tile
        sub = (i % B + j % B + k % B) % B
        blk = (i // B) * n * n + (j // B) * n + (k // B)
        unit = (ph * n * n * n + blk) * B + sub
        keys = np.concatenate([unit * n * n + pid(i, j), unit * n * n + pid(i, k), unit * n * n + pid(j, k)])
        assert np.unique(keys).size == keys.size
        tkeys = np.unique(np.stack([ph, blk]), axis=1)
        assert tkeys.shape[1] == np.unique(blk).size              # each block triple in one phase
