"""Pins of the oracle's delete-one jackknife (CPU).

The oracle recounts each resampling from scratch; these tests tie it to an
independent formulation (pairs touching the removed patch, brute force in
pure Python on tiny catalogs), to identities, and to numpy's variance.
"""
import bisect
import math

import numpy as np

import oracle
from paper_1204_6630_gb300 import synth


def _bin(dot, edges):
    theta = math.acos(min(1.0, max(-1.0, dot)))
    return bisect.bisect_right(list(edges), theta)  # number of edges <= theta


def _dot(a, b):
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]


def _tiny(seed, nd_sizes, nr_sizes):
    g = np.random.default_rng(seed)
    fp = synth.Footprint("octant")
    d = synth.clustered(sum(nd_sizes), 3, 2.0, fp, seed)
    r = synth.randoms(sum(nr_sizes), fp, seed + 1)
    doff = np.concatenate([[0], np.cumsum(nd_sizes)])
    roff = np.concatenate([[0], np.cumsum(nr_sizes)])
    edges = synth.linear_edges(0.0, 40.0, 6)
    return d, r, doff, roff, edges


def test_loo_equals_full_minus_pairs_touching_the_patch():
    d, r, doff, roff, edges = _tiny(3, [5, 0, 9, 4], [7, 3, 0, 8])
    loo, w, cov = oracle.jackknife(d, r, doff, roff, edges)
    seg_d = np.repeat(np.arange(4), np.diff(doff))
    seg_r = np.repeat(np.arange(4), np.diff(roff))
    nb2 = len(edges) + 1
    full = np.zeros((3, nb2), np.int64)
    touch = np.zeros((4, 3, nb2), np.int64)
    for i in range(len(d)):
        for j in range(i + 1, len(d)):
            k = _bin(_dot(d[i], d[j]), edges)
            full[0, k] += 1
            for p in {seg_d[i], seg_d[j]}:
                touch[p, 0, k] += 1
    for i in range(len(d)):
        for j in range(len(r)):
            k = _bin(_dot(d[i], r[j]), edges)
            full[1, k] += 1
            for p in {seg_d[i], seg_r[j]}:
                touch[p, 1, k] += 1
    for i in range(len(r)):
        for j in range(i + 1, len(r)):
            k = _bin(_dot(r[i], r[j]), edges)
            full[2, k] += 1
            for p in {seg_r[i], seg_r[j]}:
                touch[p, 2, k] += 1
    for p in range(4):
        np.testing.assert_array_equal(loo[p].astype(np.int64), full - touch[p])


def test_totals_empty_patch_and_two_patches():
    d, r, doff, roff, edges = _tiny(5, [30, 0, 25], [40, 22, 0])
    loo, w, cov = oracle.jackknife(d, r, doff, roff, edges)
    nd, nr = len(d), len(r)
    for p in range(3):
        n_p, m_p = doff[p + 1] - doff[p], roff[p + 1] - roff[p]
        a, b = nd - n_p, nr - m_p
        assert int(loo[p, 0].sum()) == a * (a - 1) // 2
        assert int(loo[p, 1].sum()) == a * b
        assert int(loo[p, 2].sum()) == b * (b - 1) // 2
    # patch 1 has no data: removing it leaves DD whole
    np.testing.assert_array_equal(loo[1, 0], oracle.count_auto(d, edges))
    # with two patches, leaving one out leaves the other alone
    d2, r2, doff2, roff2, _ = _tiny(6, [20, 15], [18, 25])
    loo2, _, _ = oracle.jackknife(d2, r2, doff2, roff2, edges)
    np.testing.assert_array_equal(loo2[0, 0], oracle.count_auto(d2[doff2[1]:], edges))
    np.testing.assert_array_equal(loo2[0, 1], oracle.count_cross(d2[doff2[1]:], r2[roff2[1]:], edges))
    np.testing.assert_array_equal(loo2[1, 2], oracle.count_auto(r2[:roff2[1]], edges))


def test_covariance_matches_numpy_variance_and_is_symmetric():
    d, r, doff, roff, edges = _tiny(7, [30, 28, 35, 31, 26], [60, 55, 70, 58, 61])
    loo, w, cov = oracle.jackknife(d, r, doff, roff, edges)
    P = len(doff) - 1
    ok = ~np.isnan(w).any(axis=0)
    np.testing.assert_allclose(np.diag(cov)[ok], np.var(w[:, ok], axis=0) * (P - 1), rtol=1e-12)
    np.testing.assert_array_equal(cov, cov.T)
    np.testing.assert_allclose(cov[np.ix_(ok, ok)], (P - 1) / P * np.cov(w[:, ok].T, bias=True) * P, rtol=1e-10)
