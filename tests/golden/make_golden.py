"""Write the hand-placed golden fixtures in this folder.

Every expected histogram here follows from exact geometry, not from any
implementation: points lie on a great circle (the equator or a meridian), so
the separation of two points is the difference of their longitudes (or
latitudes), and each separation is kept far from every bin edge compared with
the binary64 rounding of the dot product (margins are asserted below).  The
histogram convention is the paper's DD/DR/RR counts (Section 1, Eq. 1) binned
into half-open bins [t_k, t_{k+1}) with an underflow and an overflow entry:
index h = number of edges t_m <= theta.

Run:  python tests/golden/make_golden.py
"""
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEG = math.pi / 180.0


def radec(ra_deg, dec_deg):
    ra = np.asarray(ra_deg, dtype=np.float64) * DEG
    dec = np.asarray(dec_deg, dtype=np.float64) * DEG
    return np.stack([np.cos(dec) * np.cos(ra), np.cos(dec) * np.sin(ra), np.sin(dec)], axis=1)


def hist_from_separations(seps_rad, edges_rad, min_margin_rad):
    h = np.zeros(len(edges_rad) + 1, dtype=np.uint64)
    for s in seps_rad:
        margin = np.min(np.abs(edges_rad - s))
        assert margin > min_margin_rad, (s, margin)
        h[int(np.sum(edges_rad <= s))] += 1
    return h


def write(name, kind, a, b, edges, hist, header):
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line.strip() + "\n")
        f.write(f"kind {kind}\n")
        f.write("edges " + " ".join(repr(float(t)) for t in edges) + "\n")
        for tag, pts in (("a", a), ("b", b)):
            if pts is None:
                continue
            f.write(f"{tag} {len(pts)}\n")
            for p in pts:
                f.write(" ".join(repr(float(c)) for c in p) + "\n")
        f.write("hist " + " ".join(str(int(v)) for v in hist) + "\n")


def equator_ladder():
    n, step = 60, 0.3713
    edges = np.linspace(0.0, 10.0, 41) * DEG
    ra = np.arange(n) * step
    seps = [abs(ra[j] - ra[i]) * DEG for i in range(n) for j in range(i + 1, n)]
    hist = hist_from_separations(seps, edges, 1e-8)
    write("equator_ladder_linear", "auto", radec(ra, np.zeros(n)), None, edges, hist, """
    60 points on the equator at RA = 0.3713 k deg (k = 0..59); auto count (i < j).
    Pair (i, j) is separated by exactly 0.3713 |j - i| deg; 40 linear bins over 0-10 deg.
    Every separation is more than 1e-8 rad from an edge.""")


def meridian_cross_near_edges():
    # Log bins 0.01 - 10 deg; D at Dec 0 on RA 0, R on the same meridian at
    # Dec = t_k (1 +/- 1e-6) for every edge t_k: each pair sits just inside or
    # just outside an edge, well within an FP32 screen's uncertainty but
    # 1e-6 t_k >= 1.7e-10 rad from it in binary64 terms.
    edges = np.array([0.01 * 10 ** (3 * k / 64) for k in range(65)]) * DEG
    edges[0], edges[-1] = 0.01 * DEG, 10.0 * DEG
    decs = []
    for t in edges:
        decs += [t * (1 - 1e-6), t * (1 + 1e-6)]
    decs = np.array(decs) / DEG
    a = radec([0.0], [0.0])
    b = radec(np.zeros(len(decs)), decs)
    hist = hist_from_separations(decs * DEG, edges, 1e-11)
    write("meridian_cross_near_edges", "cross", a, b, edges, hist, """
    One point at (RA, Dec) = (0, 0) against points on the meridian RA = 0 at
    Dec = t_k (1 - 1e-6) and t_k (1 + 1e-6) for each of the 65 log-spaced edges
    t_k over 0.01-10 deg; cross count.  The separation is the Dec value exactly,
    so each edge gets one pair just below it and one just above it.""")


def pole_fan():
    decs = np.array([89.9953, 89.93, 89.45, 87.8, 85.3, 80.07, 70.2, 45.2, 10.7, -30.3, -89.5])
    edges = np.array([0.001, 0.01, 0.1, 1.0, 5.0, 10.0, 50.0, 100.0, 150.0]) * DEG
    a = np.array([[0.0, 0.0, 1.0]])
    b = radec(np.full(len(decs), 17.0), decs)
    hist = hist_from_separations((90.0 - decs) * DEG, edges, 1e-8)
    write("pole_fan", "cross", a, b, edges, hist, """
    The north pole against points at RA 17 deg and Dec in {89.9953 .. -89.5};
    the separation is 90 - Dec exactly; 8 bins with uneven edges; cross count.""")


def duplicates_and_antipodes():
    # Equator points at RA 10, 40, 75 deg, each twice, plus RA 190 (the antipode
    # of RA 10).  On a great circle the separation is the RA difference folded
    # to [0, 180]: 0 for duplicates, 30, 65, 35, and 180, 150, 115 to RA 190.
    ra = np.array([10.0, 40.0, 75.0, 10.0, 40.0, 75.0, 190.0])
    a = radec(ra, np.zeros(len(ra)))
    edges = np.array([0.0, 1.0, 90.0, 179.0]) * DEG
    seps = []
    for i in range(len(ra)):
        for j in range(i + 1, len(ra)):
            s = abs(ra[j] - ra[i]) % 360.0
            seps.append(min(s, 360.0 - s))
    hist = np.zeros(len(edges) + 1, dtype=np.uint64)
    for s in seps:
        hist[int(np.sum(np.degrees(edges) <= s))] += 1
    write("duplicates_and_antipodes", "auto", a, None, edges, hist, """
    Equator points at RA 10, 40, 75 deg, each twice, and RA 190 deg (antipode
    of RA 10); auto count.  Coincident pairs have theta = 0 (bin 0: the lower
    edge is inclusive); the two pairs RA 10 - RA 190 have theta = 180 deg, at
    or above the last edge 179 deg (overflow).  The other separations (30, 35,
    65, 115, 150 deg) are at least 11 deg from any edge.""")


if __name__ == "__main__":
    equator_ladder()
    meridian_cross_near_edges()
    pole_fan()
    duplicates_and_antipodes()
