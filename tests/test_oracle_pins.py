"""Pins for the CPU oracle, against facts fixed by geometry and arithmetic.

None of these retypes the oracle's formula: each expected value comes from a
closed form (exact separations of hand-placed points, pair-count identities,
the uniform-sphere bin probabilities, dyadic estimator inputs) or from a
higher-precision evaluation (mpmath) that does not use the C library's acos.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import synth

DEG = math.pi / 180.0
HERE = os.path.dirname(os.path.abspath(__file__))


def equator(ra_deg):
    ra = np.asarray(ra_deg, dtype=np.float64)
    return synth.radec_to_xyz(ra, np.zeros_like(ra))


def expected_ladder_hist(n, step_deg, edges_deg):
    """Closed form for n equator points at RA = k*step: pairs at separation
    m*step (m = 1..n-1, folded to [0, 180]) occur n - m times each."""
    h = np.zeros(len(edges_deg) + 1, dtype=np.uint64)
    for m in range(1, n):
        sep = (m * step_deg) % 360.0
        sep = min(sep, 360.0 - sep)
        h[int(np.sum(np.asarray(edges_deg) <= sep))] += n - m
    return h


# ---------------------------------------------------------------- hand-placed points
def test_equator_ladder_linear_bins():
    # Section 3: angle from the dot product and acos; separations are exact
    # multiples of the step, chosen to stay far (> 1e-6 deg) from every edge.
    n, step = 60, 0.3713
    edges_deg = np.linspace(0.0, 10.0, 41)
    seps = np.array([m * step for m in range(1, n)])
    assert np.min(np.abs(seps[:, None] - edges_deg[None, :])) > 1e-6
    got = oracle.count_auto(equator(np.arange(n) * step), edges_deg * DEG)
    np.testing.assert_array_equal(got, expected_ladder_hist(n, step, edges_deg))


def test_golden_fixtures():
    # tests/golden/*.txt: hand-placed points with counts derived from exact
    # separations (see each file's header for the derivation).
    from tests.golden import load_fixture, FIXTURES
    for name in FIXTURES:
        fx = load_fixture(name)
        if fx["kind"] == "auto":
            got = oracle.count_auto(fx["a"], fx["edges"])
        else:
            got = oracle.count_cross(fx["a"], fx["b"], fx["edges"])
        np.testing.assert_array_equal(got, fx["hist"], err_msg=name)


def test_pole_pairs_known_angles():
    # The north pole against points at declination dec: separation 90 - dec.
    decs = np.array([89.9, 85.3, 80.01, 45.2, 10.7, -30.0, -89.5])
    pole = np.array([[0.0, 0.0, 1.0]])
    pts = synth.radec_to_xyz(np.full(len(decs), 17.0), decs)
    edges_deg = np.array([0.0, 1.0, 5.0, 10.0, 50.0, 100.0, 150.0])
    got = oracle.count_cross(pole, pts, edges_deg * DEG)
    want = np.zeros(len(edges_deg) + 1, dtype=np.uint64)
    for d in decs:
        want[int(np.sum(edges_deg <= 90.0 - d))] += 1
    np.testing.assert_array_equal(got, want)


def test_antipodal_pairs_overflow_and_pi_edge():
    # Axis vectors and their negatives: the dot product is exactly -1, theta = pi,
    # which is >= the last edge pi, so these pairs are overflow.
    ax = np.eye(3)
    edges = np.array([0.0, math.pi / 2, math.pi])
    np.testing.assert_array_equal(oracle.count_cross(ax, -ax, edges), [0, 0, 6, 3])
    # Random antipodes: |v|^2 rounds to within an ulp of 1, so theta is pi or
    # within ~1e-8 of it: never below pi/2.
    v = synth.randoms(50, synth.Footprint("sphere"), seed=3)
    got = oracle.count_cross(v, -v, edges)
    assert got.sum() == 2500 and got[2] + got[3] >= 50


def test_duplicate_points_bin_zero_or_underflow():
    v = synth.randoms(20, synth.Footprint("octant"), seed=5)
    dup = np.concatenate([v, v])
    # t_0 = 0: theta = 0 lies in bin 0 (lower edge inclusive).
    e0 = np.array([0.0, 1e-3, 0.5])
    h0 = oracle.count_auto(dup, e0)
    assert h0[1] >= 20 and h0[0] == 0
    # t_0 > 0: coincident points are underflow.  A rounded |v|^2 can sit one
    # ulp below 1, putting theta at ~1.5e-8 rad, so t_0 = 1e-7 rad.
    e1 = np.array([1e-7, 1e-3, 0.5])
    h1 = oracle.count_auto(dup, e1)
    assert h1[0] == 20


def test_dot_above_one_is_clamped():
    # A unit vector whose rounded self dot product exceeds 1: acos would be
    # NaN without the clamp; with it the pair sits at theta = 0 (bin 0).
    rng = np.random.default_rng(11)
    for _ in range(100000):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        if (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2] > 1.0:
            break
    else:
        pytest.skip("no vector with rounded norm above one found")
    h = oracle.count_auto(np.stack([v, v]), np.array([0.0, 1e-6, 1.0]))
    np.testing.assert_array_equal(h, [0, 1, 0, 0])


# ---------------------------------------------------------------- identities
@pytest.mark.parametrize("n", [0, 1, 2, 3, 257])
def test_total_pair_identity(n):
    x = synth.clustered(n, 4, 1.0, synth.Footprint("octant"), seed=n) if n else np.zeros((0, 3))
    edges = synth.linear_edges(0.0, 10.0, 40)
    assert int(oracle.count_auto(x, edges).sum()) == n * (n - 1) // 2
    y = synth.randoms(31, seed=1)
    assert int(oracle.count_cross(x, y, edges).sum()) == n * 31


def test_cross_of_catalog_with_itself():
    # DR(D, D) = 2 DD(D) + N self pairs, which sit at theta ~ 0 (bin 0 here).
    x = synth.octant_small(n=600).data
    edges = synth.log_edges(0.01, 10.0, 16)
    edges0 = np.concatenate([[0.0], edges])
    dd = oracle.count_auto(x, edges0)
    dr = oracle.count_cross(x, x, edges0)
    want = 2 * dd
    want[1] += 600
    np.testing.assert_array_equal(dr, want)


def test_permutation_invariance():
    w = synth.octant_small(n=700)
    perm = np.random.default_rng(2).permutation(700)
    edges = w.edges
    np.testing.assert_array_equal(oracle.count_auto(w.data, edges),
                                  oracle.count_auto(w.data[perm], edges))
    np.testing.assert_array_equal(oracle.count_cross(w.data, w.rand, edges),
                                  oracle.count_cross(w.rand[perm], w.data, edges))


def test_threaded_rows_match_single_thread():
    w = synth.octant_small(n=900)
    np.testing.assert_array_equal(oracle.count_auto(w.data, w.edges, threads=1),
                                  oracle.count_auto(w.data, w.edges, threads=3))
    np.testing.assert_array_equal(oracle.count_cross(w.data, w.rand, w.edges, threads=1),
                                  oracle.count_cross(w.data, w.rand, w.edges, threads=4))


# ---------------------------------------------------------------- statistics
def test_uniform_sphere_bin_fractions():
    # For points uniform on the whole sphere, P(theta in [a, b)) = (cos a - cos b) / 2,
    # and pair indicators are pairwise uncorrelated (for a fixed shared point the
    # other two are independent and the conditional probability is still p), so
    # var(count) = M p (1 - p) with M = N (N - 1) / 2.
    n = 6000
    x = synth.randoms(n, synth.Footprint("sphere"), seed=7)
    edges = np.linspace(0.0, math.pi, 13)
    h = oracle.count_auto(x, edges, threads=4)
    m = n * (n - 1) / 2
    p = (np.cos(edges[:-1]) - np.cos(edges[1:])) / 2
    z = (h[1:-1] - m * p) / np.sqrt(m * p * (1 - p))
    assert np.all(np.abs(z) < 5.0), z
    assert h[0] == 0 and h[-1] == 0


def test_estimator_near_zero_for_unclustered_data():
    # D and R independent uniform draws on the same footprint: w ~ 0.
    fp = synth.Footprint("octant")
    d = synth.randoms(3000, fp, seed=21)
    r = synth.randoms(3000, fp, seed=22)
    edges = synth.linear_edges(2.0, 20.0, 6)
    _, _, _, w = oracle.correlation(d, r, edges, threads=4)
    assert np.all(np.abs(w) < 0.05), w


def test_estimator_detects_clustering():
    w = synth.octant_small(n=3000)
    _, _, _, wt = oracle.correlation(w.data, w.rand, synth.linear_edges(0.0, 2.0, 4), threads=4)
    assert wt[0] > 1.0


# ---------------------------------------------------------------- estimator closed forms
def test_estimator_exact_dyadic_cases():
    # nd = 4 -> 6 DD pairs; nr = 5 -> 10 RR pairs; 20 DR pairs.
    dd = [6, 3, 0, 6]
    dr = [15, 10, 5, 20]
    rr = [10, 5, 10, 0]
    w = oracle.estimate(dd, dr, rr, 4, 5, oracle.LS_EXACT)
    # bin 0: nDD=1, nDR=0.75, nRR=1 -> (1 - 1.5 + 1)/1 = 0.5
    # bin 1: nDD=0.5, nDR=0.5, nRR=0.5 -> (0.5 - 1 + 0.5)/0.5 = 0
    # bin 2: nDD=0, nDR=0.25, nRR=1 -> (0 - 0.5 + 1)/1 = 0.5
    # bin 3: RR = 0 -> NaN
    assert w[0] == 0.5 and w[1] == 0.0 and w[2] == 0.5 and math.isnan(w[3])


def test_estimator_paper_reading_dyadic():
    # Eq. 1 as printed: w = 1 + q^2 DD'/RR' - 2 q DR/RR', q = nr/nd,
    # DD' = 2 DD and RR' = 2 RR (ordered pairs).  nd = 4, nr = 8 -> q = 2.
    dd, dr, rr = [2], [8], [4]
    w = oracle.estimate(dd, dr, rr, 4, 8, oracle.LS_PAPER)
    # 1 + 4 * (4/8) - 4 * (8/8) = 1 + 2 - 4 = -1
    assert w[0] == -1.0


def test_estimators_agree_to_order_one_over_n():
    w = synth.octant_small(n=2000)
    dd, dr, rr, we = oracle.correlation(w.data, w.rand, synth.linear_edges(0.0, 5.0, 5), threads=4)
    wp = oracle.estimate(dd[1:-1], dr[1:-1], rr[1:-1], 2000, 2000, oracle.LS_PAPER)
    # Same catalogs sizes: the two readings differ only through N/(N-1) factors.
    assert np.all(np.abs((1 + we) - (1 + wp)) <= 3.0 / 2000 * np.abs(1 + we) + 1e-12)


# ---------------------------------------------------------------- independent brute force
def test_tiny_brute_force_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    x = synth.clustered(48, 3, 2.0, synth.Footprint("octant"), seed=9)
    edges = synth.log_edges(0.05, 60.0, 12)
    want = np.zeros(len(edges) + 1, dtype=np.uint64)
    e_mp = [mp.mpf(float(t)) for t in edges]
    near = 0
    for i in range(len(x)):
        for j in range(i + 1, len(x)):
            a, b = x[i], x[j]
            d = (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]   # numpy float64: one rounding per op
            d = min(1.0, max(-1.0, float(d)))
            th = mp.acos(mp.mpf(d))
            if min(abs(th - t) for t in e_mp) < mp.mpf("1e-12"):
                near += 1
            want[sum(1 for t in e_mp if t <= th)] += 1
    assert near == 0
    np.testing.assert_array_equal(oracle.count_auto(x, edges), want)
