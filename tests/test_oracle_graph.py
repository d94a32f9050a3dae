"""Pins of the oracle's radius graph: a k-d tree (scipy cKDTree, float64) on
poses without near-cutoff pairs gives the same edge sets; boundary pairs follow
the strict-inequality rule; structure (symmetric, sorted, no self loops)."""

import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import fusion_oracle as O
from synth import poses


def _pairs(rp, col):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return set(zip(rows.tolist(), col.tolist()))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_edges_match_kdtree(seed):
    xyz, feat, n_lig = poses.make_pose(seed, (15, 60), (250, 800))
    g = O.radius_graph(xyz, 1.6, 4.5)
    t = cKDTree(xyz.astype(np.float64))
    within_nc = t.query_pairs(4.5, output_type="ndarray")
    within_cov = t.query_pairs(1.6, output_type="ndarray")
    # query_pairs uses <=; the generator keeps every pair 1e-5 A^2 away from the cutoffs
    cov = {(int(i), int(j)) for i, j in within_cov} | {(int(j), int(i)) for i, j in within_cov}
    allp = {(int(i), int(j)) for i, j in within_nc} | {(int(j), int(i)) for i, j in within_nc}
    assert _pairs(*g["cov"]) == cov
    assert _pairs(*g["nc"]) == allp - cov


def test_graph_structure():
    xyz, feat, n_lig = poses.make_pose(11, (20, 50), (300, 600))
    g = O.radius_graph(xyz, 1.6, 4.5)
    for name in ("cov", "nc"):
        rp, col = g[name]
        P = _pairs(rp, col)
        assert all((j, i) in P for i, j in P)
        assert all(i != j for i, j in P)
        for i in range(len(rp) - 1):
            r = col[rp[i]:rp[i + 1]]
            assert np.all(np.diff(r) > 0)
    assert not (_pairs(*g["cov"]) & _pairs(*g["nc"]))


def test_boundary_pairs_use_strict_inequality():
    c = np.float32(1.6)
    xyz = np.array([[0, 0, 0], [c, 0, 0], [10, 0, 0], [10, 4.5, 0], [20, 0, 0], [20, 1.0, 0]], dtype=np.float32)
    g = O.radius_graph(xyz, 1.6, 4.5)
    cov = _pairs(*g["cov"])
    nc = _pairs(*g["nc"])
    # exactly at the covalent cutoff: not covalent, but non-covalent
    assert (0, 1) not in cov and (0, 1) in nc
    # exactly at the non-covalent cutoff: no edge
    assert (2, 3) not in cov and (2, 3) not in nc
    # well inside: covalent only
    assert (4, 5) in cov and (4, 5) not in nc


def test_isolated_atoms_and_single_atom():
    xyz = np.array([[0, 0, 0], [100, 0, 0]], dtype=np.float32)
    g = O.radius_graph(xyz, 1.6, 4.5)
    assert g["cov"][0].tolist() == [0, 0, 0] and g["nc"][0].tolist() == [0, 0, 0]
    g1 = O.radius_graph(xyz[:1], 1.6, 4.5)
    assert len(g1["nc"][1]) == 0
