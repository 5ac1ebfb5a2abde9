"""Spatial pruning (TPCF_F_PRUNE): blocks of pairs whose bounding spheres are
provably beyond the last edge are skipped, and every histogram stays equal
to the oracle's and to the unpruned kernel's: octant and full-sphere
catalogs, clusters placed right at the pruning distance, vectors off unit
norm, patches and the jackknife, the 3-D variant, and ranges that cannot
prune (last edge at pi)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import build, synth

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1204_6630_gb300 import tpcf
    tpcf.load()
    return tpcf


def oracle_all(d, r, edges, euclid=False):
    return (oracle.count_auto(d, edges, THREADS, euclid=euclid),
            oracle.count_cross(d, r, edges, THREADS, euclid=euclid),
            oracle.count_auto(r, edges, THREADS, euclid=euclid))


def run(T, d, r, edges, prune, euclid=False, **kw):
    flags = T.TPCF_F_PRUNE if prune else 0
    with T.Context(flags=flags, **kw) as ctx:
        if euclid:
            cd, cr, b = ctx.catalog3d(d), ctx.catalog3d(r), ctx.bins3d(edges)
        else:
            cd, cr, b = ctx.catalog(d), ctx.catalog(r), ctx.bins(edges)
        got, st = ctx.count_all(cd, cr, b, stats=True)
    assert st["device_error"] == 0
    return got, st


def test_octant_small_against_oracle(T):
    w = synth.octant_small(seed=0)
    want = oracle_all(w.data, w.rand, w.edges)
    got, st = run(T, w.data, w.rand, w.edges, True)
    for g, o in zip(got, want):
        np.testing.assert_array_equal(g, o)
    assert st["pruned_pairs"] > 0
    _, st0 = run(T, w.data, w.rand, w.edges, False)
    assert st0["pruned_pairs"] == 0


@pytest.mark.parametrize("shape", [dict(threads=128, ipt=8), dict(threads=512, ipt=8), dict(threads=256, ipt=16)])
def test_small_range_full_sphere_every_shape(T, shape):
    # a 2 deg range on the full sphere: nearly every block prunes
    d = synth.clustered(30000, 64, 0.3, synth.Footprint("sphere"), seed=4)
    r = synth.randoms(40000, synth.Footprint("sphere"), seed=5)
    edges = synth.log_edges(0.01, 2.0, 30)
    d_s, r_s = d[:6000], r[:7000]
    got, st = run(T, d_s, r_s, edges, True, **shape)
    for g, o in zip(got, oracle_all(d_s, r_s, edges)):
        np.testing.assert_array_equal(g, o)
    big, stb = run(T, d, r, edges, True, **shape)
    ref, _ = run(T, d, r, edges, False, **shape)
    for g, o in zip(big, ref):
        np.testing.assert_array_equal(g, o)
    assert stb["pruned_pairs"] > 0.6 * stb["pairs"]  # (512-point warps at ipt 16: coarser spheres)


def _cap_points(centre, radius_rad, n, rng):
    """n unit vectors within radius_rad of the unit vector centre."""
    c = centre / np.linalg.norm(centre)
    a = np.array([1.0, 0.0, 0.0]) if abs(c[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(c, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(c, e1)
    rho = radius_rad * np.sqrt(rng.random(n))
    phi = rng.random(n) * 2 * np.pi
    v = (np.cos(rho)[:, None] * c + np.sin(rho)[:, None] * (np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2))
    return v / np.linalg.norm(v, axis=1)[:, None]


@pytest.mark.parametrize("gap_deg", [-0.02, -1e-4, 0.0, 1e-4, 0.02])
def test_clusters_at_the_pruning_distance(T, gap_deg):
    # two tight clusters whose nearest points are about t_B apart: pairs right at
    # the last edge must be counted exactly whether or not the blocks prune
    rng = np.random.default_rng(11)
    tB = 3.0
    rad = math.radians(0.05)
    sep = math.radians(tB + gap_deg) + 2 * rad
    c1 = np.array([1.0, 0.0, 0.0])
    c2 = np.array([math.cos(sep), math.sin(sep), 0.0])
    d = _cap_points(c1, rad, 512, rng)
    r = np.concatenate([_cap_points(c2, rad, 512, rng), _cap_points(c1, rad, 256, rng)])
    edges = synth.linear_edges(0.0, tB, 30)
    got, _ = run(T, d, r, edges, True, threads=128, ipt=8)
    for g, o in zip(got, oracle_all(d, r, edges)):
        np.testing.assert_array_equal(g, o)


def test_vectors_off_unit_norm(T):
    # norms 1 +- 5e-7 (inside the catalog tolerance): the pruning bound allows for them
    rng = np.random.default_rng(3)
    d = synth.clustered(5000, 32, 0.4, seed=6)
    r = synth.randoms(6000, seed=7)
    d = d * (1.0 + rng.uniform(-5e-7, 5e-7, (len(d), 1)))
    r = r * (1.0 + rng.uniform(-5e-7, 5e-7, (len(r), 1)))
    edges = synth.linear_edges(0.0, 4.0, 20)
    got, st = run(T, d, r, edges, True)
    for g, o in zip(got, oracle_all(d, r, edges)):
        np.testing.assert_array_equal(g, o)
    assert st["pruned_pairs"] > 0


def test_last_edge_at_pi_never_prunes(T):
    w = synth.octant_small(seed=2, n=3000)
    edges = synth.linear_edges(0.0, 180.0, 12)  # radians, last edge pi
    got, st = run(T, w.data, w.rand, edges, True)
    assert st["pruned_pairs"] == 0
    for g, o in zip(got, oracle_all(w.data, w.rand, edges)):
        np.testing.assert_array_equal(g, o)


def test_octant_precision_full_size_equals_unpruned(T):
    import torch
    w = synth.octant_precision(seed=0)
    dd_, dr_ = torch.from_numpy(w.data).cuda(), torch.from_numpy(w.rand).cuda()
    got, st = run(T, dd_, dr_, w.edges, True)
    ref, st0 = run(T, dd_, dr_, w.edges, False)
    for g, o in zip(got, ref):
        np.testing.assert_array_equal(g, o)
    assert st["pairs"] == st0["pairs"] and st["pruned_pairs"] > 0.5 * st["pairs"]
    assert st["band_pairs"] == st0["band_pairs"]


def test_patches_and_jackknife_equal_unpruned(T):
    d, r, doff, roff = synth.jackknife_patches(seed=1, nd=60000, npatch=24)
    edges = synth.linear_edges(0.0, 5.0, 20)
    out = []
    for prune in (False, True):
        with T.Context(flags=T.TPCF_F_PRUNE if prune else 0) as ctx:
            cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
            h = ctx.count_patches(cd, cr, b)
            loo, wv, cov = ctx.jackknife(cd, cr, b)
            out.append((h, loo, wv, cov))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_array_equal(out[0][3], out[1][3])


@pytest.mark.parametrize("offset", [0.0, 1e6])
def test_3d_against_oracle_and_unpruned(T, offset):
    d = synth.box_clustered(6000, 40, 2.0, 400.0, 2) + offset
    r = synth.box_points(8000, 400.0, 3) + offset
    edges = synth.log_edges_r(0.5, 30.0, 20)
    got, st = run(T, d, r, edges, True, euclid=True)
    for g, o in zip(got, oracle_all(d, r, edges, euclid=True)):
        np.testing.assert_array_equal(g, o)
    assert st["pruned_pairs"] > 0
    d2 = synth.box_clustered(150000, 400, 2.0, 1000.0, 4) + offset
    r2 = synth.box_points(150000, 1000.0, 5) + offset
    a, _ = run(T, d2, r2, edges, True, euclid=True)
    b, _ = run(T, d2, r2, edges, False, euclid=True)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_3d_huge_coordinates(T):
    # coordinates near 1e27 (separations up to 3e27: the spheres live in a
    # 2^-64-scaled space), edges up to the 1e18 limit
    rng = np.random.default_rng(9)
    d = rng.uniform(-1e27, 1e27, (3000, 3))
    r = np.concatenate([d[:500] + rng.normal(0, 3e17, (500, 3)), rng.uniform(-1e27, 1e27, (2500, 3))])
    edges = np.array([0.0, 1e16, 1e17, 3e17, 1e18])
    got, _ = run(T, d, r, edges, True, euclid=True)
    for g, o in zip(got, oracle_all(d, r, edges, euclid=True)):
        np.testing.assert_array_equal(g, o)


def test_server_jobs_with_pruning(T):
    # jobs served by a pruning context == the oracle
    specs = sorted(synth.serving_jobs(60, seed=3), key=lambda s: s["nd"])[:6]
    jobs = [synth.materialise_job(s) for s in specs]
    with T.Context(flags=T.TPCF_F_PRUNE, server_workers=3) as ctx:
        ids = [ctx.submit(w.data, w.rand, w.edges) for w in jobs]
        for jid, w in zip(ids, jobs):
            res = ctx.poll(jid, len(w.edges))
            dd, dr, rr = oracle_all(w.data, w.rand, w.edges)
            np.testing.assert_array_equal(res["dd"], dd)
            np.testing.assert_array_equal(res["dr"], dr)
            np.testing.assert_array_equal(res["rr"], rr)
