"""Soundness of the spatial-pruning test, on the CPU.

Bounding spheres are built as the catalog preparation builds them (the
FP32-rounded mean of a group's points as centre, the binary64 distance to the
farthest point enlarged by 2^-20 and rounded up to FP32 as radius), a warp's
sphere is combined from its groups' spheres, and the block test is evaluated
in FP32 with the kernel's 2^-20 margins against the host's threshold.  Every
block the test skips must hold only overflow pairs by the oracle's count.
Blocks are placed at random and adversarially (their nearest points within
1e-9..1e-3 rad of the last edge), with norms off unity and, in 3-D, with
coordinates up to 1e27.
"""
import math

import numpy as np

import oracle
from paper_1204_6630_gb300 import tpcf

M = np.float32(2.0 ** -20)
SCALE_3D = 2.0 ** -64


def _ru32(x: float) -> np.float32:
    f = np.float32(x)
    return f if float(f) >= x else np.nextafter(f, np.float32(np.inf))


def _group_sphere(p: np.ndarray, scale: float) -> np.ndarray:
    q = p * scale
    c = (q.sum(axis=0) / len(q)).astype(np.float32)
    r = float(np.sqrt(((q - c.astype(np.float64)) ** 2).sum(axis=1)).max())
    return np.array([c[0], c[1], c[2], _ru32(r * (1.0 + 2.0 ** -20))], np.float32)


def _warp_sphere(spheres: list[np.ndarray]) -> np.ndarray:
    g = np.array(spheres, np.float32)
    inv = np.float32(1.0) / np.float32(len(g))
    c = np.array([g[:, 0].sum(dtype=np.float32) * inv, g[:, 1].sum(dtype=np.float32) * inv,
                  g[:, 2].sum(dtype=np.float32) * inv], np.float32)
    d = np.sqrt(((c[None, :] - g[:, :3]) ** 2).sum(axis=1, dtype=np.float32)).astype(np.float32)
    r = np.max(d + g[:, 3]).astype(np.float32)
    return np.array([c[0], c[1], c[2], r * (np.float32(1.0) + M)], np.float32)


def _prunes(a: np.ndarray, b: np.ndarray, thr: np.float32) -> bool:
    d = (a[:3] - b[:3]).astype(np.float32)
    D = np.sqrt(np.float32(d[2] * d[2]) + np.float32(np.float32(d[1] * d[1]) + np.float32(d[0] * d[0])))
    L = np.float32(D * (np.float32(1.0) - M)) - np.float32((a[3] + b[3]) * (np.float32(1.0) + M))
    return bool(L > thr)


def _cap(centre, radius, n, rng, norm_jitter=0.0):
    c = centre / np.linalg.norm(centre)
    a = np.array([1.0, 0.0, 0.0]) if abs(c[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(c, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(c, e1)
    rho = radius * np.sqrt(rng.random(n))
    phi = rng.random(n) * 2 * np.pi
    v = np.cos(rho)[:, None] * c + np.sin(rho)[:, None] * (np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2)
    v /= np.linalg.norm(v, axis=1)[:, None]
    if norm_jitter:
        v *= 1.0 + rng.uniform(-norm_jitter, norm_jitter, (n, 1))
    return v


def _angular_thr(edges, cats) -> np.float32:
    c_b = tpcf.tpcf_bins_thresholds(edges)[0][-1]
    eps = max(float(np.abs((x * x).sum(axis=1) - 1.0).max()) for x in cats) + 4e-16
    return _ru32(math.sqrt(max(0.0, 2.0 * (1.0 + eps) - 2.0 * (c_b - 1e-15))))


def test_angular_blocks_near_the_pruning_distance():
    rng = np.random.default_rng(1)
    edges = np.radians(np.linspace(0.0, 3.0, 16))
    t_b = edges[-1]
    skipped = 0
    for trial in range(300):
        rad = 10 ** rng.uniform(-5, -2)
        jitter = 5e-7 if trial % 3 == 0 else 0.0
        gap = [-1e-3, -1e-6, -1e-9, 0.0, 1e-9, 1e-6, 1e-3][trial % 7] * rng.random()
        sep = t_b + 2 * rad + gap
        ca = rng.normal(size=3)
        ca /= np.linalg.norm(ca)
        ortho = np.cross(ca, rng.normal(size=3))
        ortho /= np.linalg.norm(ortho)
        cb = math.cos(sep) * ca + math.sin(sep) * ortho
        wa = [_cap(ca, rad, 128, rng, jitter), _cap(ca, rad, 128, rng, jitter)]  # a warp: two groups
        jb = _cap(cb, rad, 128, rng, jitter)
        thr = _angular_thr(edges, wa + [jb])
        if _prunes(_warp_sphere([_group_sphere(g, 1.0) for g in wa]), _group_sphere(jb, 1.0), thr):
            skipped += 1
            h = oracle.count_cross(np.concatenate(wa), jb, edges)
            assert int(h[-1]) == 256 * 128, (trial, sep, rad, gap, h)
    assert skipped > 20  # the test does skip blocks beyond the range


def test_angular_random_blocks_on_the_sphere():
    rng = np.random.default_rng(2)
    edges = np.radians(np.geomspace(0.01, 10.0, 20))
    edges = np.concatenate([[0.0], edges])
    for _ in range(100):
        ca, cb = rng.normal(size=(2, 3))
        rad = 10 ** rng.uniform(-3, -0.5)
        wa = [_cap(ca, rad, 128, rng), _cap(ca, rad, 128, rng)]
        jb = _cap(cb, rad, 128, rng)
        thr = _angular_thr(edges, wa + [jb])
        if _prunes(_warp_sphere([_group_sphere(g, 1.0) for g in wa]), _group_sphere(jb, 1.0), thr):
            assert int(oracle.count_cross(np.concatenate(wa), jb, edges)[-1]) == 256 * 128


def test_3d_blocks_near_the_pruning_distance_and_huge_coordinates():
    rng = np.random.default_rng(3)
    skipped = 0
    for trial in range(300):
        base = 10 ** rng.uniform(0, 27)
        r_b = min(1e18, base * 10 ** rng.uniform(-3, 0))
        edges = np.array([0.0, r_b / 4, r_b / 2, r_b])
        s_b = tpcf.tpcf_bins_thresholds_3d(edges)[0][-1]
        thr = _ru32(math.sqrt(s_b) * (1.0 + 1e-12) * SCALE_3D)
        rad = r_b * 10 ** rng.uniform(-4, 0)
        gap = r_b * [-1e-3, -1e-7, 0.0, 1e-7, 1e-3, 1.0][trial % 6] * rng.random()
        ca = rng.uniform(-base, base, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        cb = ca + u * (r_b + 2 * rad + gap)

        def ball(c):
            v = rng.normal(size=(128, 3))
            v *= (rad * rng.random((128, 1)) ** (1 / 3)) / np.linalg.norm(v, axis=1)[:, None]
            return c + v

        wa = [ball(ca), ball(ca)]
        jb = ball(cb)
        if _prunes(_warp_sphere([_group_sphere(g, SCALE_3D) for g in wa]), _group_sphere(jb, SCALE_3D), thr):
            skipped += 1
            h = oracle.count_cross(np.concatenate(wa), jb, edges, euclid=True)
            assert int(h[-1]) == 256 * 128, (trial, base, r_b, rad, gap, h)
    assert skipped > 30


def test_coincident_groups_at_the_last_edge():
    # groups of one repeated point (radius = the FP32 rounding of the centre): the
    # sphere gap is the pair's own distance, so the margins alone keep an in-range
    # pair at t_B - delta from being skipped (a margin-less test skips it)
    rng = np.random.default_rng(4)
    edges = np.radians(np.linspace(0.0, 3.0, 16))
    t_b = edges[-1]
    for delta in (1e-4, 1e-6, 1e-8, 1e-10, -1e-10, -1e-8, -1e-6, -1e-4):
        for _ in range(20):
            a = rng.normal(size=3)
            a /= np.linalg.norm(a)
            ortho = np.cross(a, rng.normal(size=3))
            ortho /= np.linalg.norm(ortho)
            b = math.cos(t_b - delta) * a + math.sin(t_b - delta) * ortho
            wa = [np.repeat(a[None, :], 128, 0), np.repeat(a[None, :], 128, 0)]
            jb = np.repeat(b[None, :], 128, 0)
            thr = _angular_thr(edges, wa + [jb])
            if _prunes(_warp_sphere([_group_sphere(g, 1.0) for g in wa]), _group_sphere(jb, 1.0), thr):
                assert int(oracle.count_cross(np.concatenate(wa), jb, edges)[-1]) == 256 * 128, delta


def test_coincident_groups_at_the_last_3d_edge():
    rng = np.random.default_rng(5)
    for base in (1.0, 1e6, 1e20, 1e27):
        r_b = min(1e18, base)
        edges = np.array([0.0, r_b / 2, r_b])
        s_b = tpcf.tpcf_bins_thresholds_3d(edges)[0][-1]
        thr = _ru32(math.sqrt(s_b) * (1.0 + 1e-12) * SCALE_3D)
        for rel in (1e-3, 1e-6, 1e-9, -1e-9, -1e-6, -1e-3):
            for _ in range(10):
                a = rng.uniform(-base, base, 3)
                u = rng.normal(size=3)
                u /= np.linalg.norm(u)
                b = a + u * r_b * (1.0 - rel)
                wa = [np.repeat(a[None, :], 128, 0), np.repeat(a[None, :], 128, 0)]
                jb = np.repeat(b[None, :], 128, 0)
                if _prunes(_warp_sphere([_group_sphere(g, SCALE_3D) for g in wa]), _group_sphere(jb, SCALE_3D), thr):
                    h = oracle.count_cross(np.concatenate(wa), jb, edges, euclid=True)
                    assert int(h[-1]) == 256 * 128, (base, rel)
