"""Pins of the oracle's 3-D variant (Euclidean separations, Section 1's
spatial two-point function): exact distances of hand-placed points, totals,
a pure-Python brute force, and the textbook distance distribution of
uniform points in a cube."""
import math

import numpy as np
import pytest

import oracle


def test_pythagorean_points_land_on_the_bins_their_exact_distances_give():
    # distances 3, 5, 7 and 9 exactly (Pythagorean quadruples), all on bin edges
    pts = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0], [3.0, 4.0, 0.0], [2.0, 3.0, 6.0], [1.0, 4.0, 8.0]])
    edges = np.array([0.5, 3.0, 5.0, 7.0, 9.0, 100.0])
    h = oracle.count_auto(pts, edges, euclid=True)
    # pairs from the origin: r = 3, 5, 7, 9 -> bins [3,5), [5,7), [7,9), [9,100)
    want = np.zeros(len(edges) + 1, np.uint64)
    for i in range(len(pts)):
        for j in range(i + 1, len(pts)):
            d = pts[i] - pts[j]
            r = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
            want[sum(1 for e in edges if e <= r)] += 1
    np.testing.assert_array_equal(h, want)
    assert h[2] >= 1 and h[3] >= 1 and h[4] >= 1 and h[5] >= 1  # each exact distance in its upper bin
    # a duplicate point has r = 0: underflow unless an edge is at 0
    dup = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0]])
    assert oracle.count_auto(dup, np.array([0.5, 1.0]), euclid=True)[0] == 1
    assert oracle.count_auto(dup, np.array([0.0, 1.0]), euclid=True)[1] == 1


def test_totals_and_pure_python_brute_force():
    g = np.random.default_rng(3)
    d = g.uniform(-50, 50, (40, 3))
    r = g.uniform(-50, 50, (35, 3)) * np.array([1.0, 0.5, 2.0])
    edges = np.array([0.0, 5.0, 12.5, 30.0, 60.0])
    dd = oracle.count_auto(d, edges, euclid=True)
    dr = oracle.count_cross(d, r, edges, euclid=True)
    assert int(dd.sum()) == 40 * 39 // 2 and int(dr.sum()) == 40 * 35
    want = np.zeros(len(edges) + 1, np.uint64)
    for a in d:
        for b in r:
            x, y, z = float(a[0]) - float(b[0]), float(a[1]) - float(b[1]), float(a[2]) - float(b[2])
            rr = math.sqrt((x * x + y * y) + z * z)
            want[sum(1 for e in edges if e <= rr)] += 1
    np.testing.assert_array_equal(dr, want)
    # translation and axis permutation leave separations unchanged (up to rounding on edges)
    shifted = oracle.count_auto(d + 1024.0, edges, euclid=True)  # exact shift by a power of two
    np.testing.assert_array_equal(shifted, dd)


@pytest.mark.parametrize("seed", [0, 1])
def test_uniform_cube_distance_distribution(seed):
    # density of the distance s between two uniform points of the unit cube, 0 <= s <= 1:
    # p(s) = s^2 (4 pi - 6 pi s + 8 s^2 - s^3)
    F = lambda x: 4 * math.pi * x ** 3 / 3 - 6 * math.pi * x ** 4 / 4 + 8 * x ** 5 / 5 - x ** 6 / 6
    L, n = 200.0, 3000
    pts = np.random.default_rng(seed).uniform(0.0, L, (n, 3))
    edges = np.array([10.0, 20.0, 40.0, 80.0, 140.0, 200.0])
    h = oracle.count_auto(pts, edges, threads=4, euclid=True)
    npairs = n * (n - 1) // 2
    for k in range(len(edges) - 1):
        p = F(edges[k + 1] / L) - F(edges[k] / L)
        sigma = math.sqrt(npairs * p * (1 - p) * 4.0)  # binomial, inflated for pairs sharing points
        assert abs(int(h[k + 1]) - npairs * p) < 6 * sigma, (k, int(h[k + 1]), npairs * p)
