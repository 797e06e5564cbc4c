"""The relabeled-oracle helper maps the oracle's state back to the caller's
labels correctly: Dykstra's invariant v = v0 - W^-1 A^T y/eps holds for the
mapped state against the ORIGINAL instance's dense rows (a wrong pair, triplet
or row mapping breaks it)."""
import numpy as np
import pytest

from oracle import dense
from instances import planted_partition
from relabel import RelabeledOracle, deal_labels


@pytest.mark.parametrize("n,B", [(3, 8), (10, 4), (13, 8), (20, 8), (23, 16)])
def test_deal_labels_is_a_permutation_spreading_neighbours(n, B):
    lab = deal_labels(n, B)
    assert sorted(lab.tolist()) == list(range(n))
    nb = -(-n // B)
    blocks = lab // B
    # the first nb objects land in nb different blocks
    assert len(set(blocks[:nb].tolist())) == min(nb, n)


@pytest.mark.parametrize("n,B,sweeps", [(9, 4, 2), (12, 8, 3), (17, 8, 1)])
def test_mapped_state_satisfies_the_invariant_on_the_original_instance(n, B, sweeps):
    d, w, _ = planted_partition(n, 3, 0.6, 0.3, seed=n, weights=(0.5, 2.0))
    r = RelabeledOracle(n, d, w, 0.3, B)
    r.sweep(sweeps)
    assert dense.invariant_residual(n, d, w, 0.3, r.x, r.f, r.ytri, r.ypair) <= 1e-12
    assert r.ytri.max() > 0 or r.ypair.max() > 0
