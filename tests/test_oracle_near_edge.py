"""The oracle's enumeration of pairs whose angle lies within 1e-12 rad of a
bin edge (the only pairs whose bin may depend on which arc-cosine decides
it), pinned by hand-placed pairs at known offsets from the edges, and run on
the 8192 + 8192 octant workload in full, where it finds none."""
import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import synth


def _equator(phis):
    phis = np.asarray(phis, dtype=np.float64)
    return np.stack([np.cos(phis), np.sin(phis), np.zeros_like(phis)], axis=1)


def test_hand_placed_pairs_at_known_offsets():
    # pairs (origin, point at angle t_k + delta) on the equator: the oracle's
    # angle is within ~4e-16 of t_k + delta (acos of a correctly rounded cosine)
    edges = np.array([0.0, 0.1, 0.25, 0.5, 1.0])
    near = [0.1 + 3e-13, 0.25 - 4e-13, 0.5 + 1e-13, 1.0 - 2e-13]
    far = [0.1 + 5e-12, 0.25 - 3e-12, 0.5 + 2e-11, 0.75, 0.05]
    a = _equator([0.0])
    b = _equator(near + far)
    count, pairs = oracle.near_edge_pairs(a, b, edges, auto=False)
    assert count == len(near)
    got = sorted(j for _, j, _ in pairs)
    assert got == list(range(len(near)))
    for _, j, gap in pairs:
        want = near[j] - edges[np.argmin(np.abs(edges - near[j]))]
        assert abs(gap - want) < 1e-15
    # a tolerance of 0 finds nothing; a wider one also finds the far pairs within it
    assert oracle.near_edge_pairs(a, b, edges, auto=False, tol=0.0)[0] == 0
    assert oracle.near_edge_pairs(a, b, edges, auto=False, tol=1e-11)[0] == len(near) + 2


def test_auto_mode_visits_each_unordered_pair_once():
    edges = np.array([0.0, 0.2, 0.4])
    x = _equator([0.0, 0.2 + 1e-13, 0.4 + 2e-13, 0.2 - 5e-13])
    # near pairs: (0,1) at 0.2, (0,2) at 0.4, (0,3) at 0.2, (1,2) at 0.2, (2,3) at 0.2 (+7e-13),
    # and (1,3), 6e-13 apart, at the edge 0 (its cosine rounds to 1: the angle is exactly 0)
    count, pairs = oracle.near_edge_pairs(x, None, edges, auto=True)
    assert count == 6
    assert sorted((i, j) for i, j, _ in pairs) == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    assert all(i < j for i, j, _ in pairs)


def test_octant_small_workload_has_no_pair_within_1e12_of_an_edge():
    w = synth.octant_small(seed=0, n=8192)
    total = 0
    for auto, a, b in ((True, w.data, None), (True, w.rand, None), (False, w.data, w.rand)):
        c, _ = oracle.near_edge_pairs(a, b, w.edges, auto, tol=1e-12, threads=8)
        total += c
    assert total == 0
