"""The 3-D variant (Euclidean separations) on the GPU against the oracle's
3-D counts: exact distances on bin edges, clustered boxes, large coordinates,
duplicates, ragged sizes and every kernel shape, both precisions, patches and
the jackknife, and invalid mixes of angular and 3-D objects."""
import os

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import build, synth

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
SCREEN, PLAIN = 0, 1


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1204_6630_gb300 import tpcf
    tpcf.load()
    return tpcf


def o3(d, r, edges):
    return (oracle.count_auto(d, edges, THREADS, euclid=True), oracle.count_cross(d, r, edges, THREADS, euclid=True),
            oracle.count_auto(r, edges, THREADS, euclid=True))


def g3(ctx, d, r, edges):
    return ctx.count_all(ctx.catalog3d(d), ctx.catalog3d(r), ctx.bins3d(edges))


def test_exact_distances_on_edges(T):
    # integer points: many distances are integers that sit exactly on the edges
    g = np.random.default_rng(1)
    d = g.integers(-6, 7, (700, 3)).astype(np.float64)
    r = g.integers(-6, 7, (900, 3)).astype(np.float64)
    edges = np.array([0.0, 1.0, 2.0, 3.0, 5.0, 7.0, 9.0, 11.0, 13.0])
    with T.Context() as ctx:
        got = g3(ctx, d, r, edges)
    for a, b in zip(got, o3(d, r, edges)):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", [SCREEN, PLAIN])
@pytest.mark.parametrize("side,offset", [(100.0, 0.0), (1000.0, 0.0), (50.0, 1e6)])
def test_clustered_boxes(T, precision, side, offset):
    d = synth.box_clustered(5000, 40, side / 200, side, 2) + offset
    r = synth.box_points(7000, side, 3) + offset
    for edges in (synth.log_edges_r(side / 2000, side / 5, 24), np.linspace(0.0, side / 3, 17)):
        with T.Context(precision=precision) as ctx:
            got, st = ctx.count_all(ctx.catalog3d(d), ctx.catalog3d(r), ctx.bins3d(edges), stats=True)
        assert st["device_error"] == 0
        for a, b in zip(got, o3(d, r, edges)):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("shape", [(128, 8), (256, 8), (512, 8), (256, 16)])
def test_ragged_sizes_and_shapes(T, shape):
    edges = synth.log_edges_r(0.2, 40.0, 12)
    for n in (0, 1, 2, 255, 257, 4097):
        d = synth.box_clustered(n, 5, 1.0, 60.0, n + 7)
        r = synth.box_points(n // 2 + 3, 60.0, n + 9)
        with T.Context(threads=shape[0], ipt=shape[1]) as ctx:
            got = g3(ctx, d, r, edges)
        for a, b in zip(got, o3(d, r, edges)):
            np.testing.assert_array_equal(a, b, err_msg=f"n={n} shape={shape}")


def test_duplicates_and_zero_edge(T):
    base = synth.box_points(300, 10.0, 4)
    d = np.concatenate([base, base[:100], np.repeat(base[:1], 50, axis=0)])
    for edges in (np.array([0.0, 0.5, 2.0]), np.array([1e-9, 0.5, 2.0])):
        with T.Context() as ctx:
            got = g3(ctx, d, d[:120], edges)
        for a, b in zip(got, o3(d, d[:120], edges)):
            np.testing.assert_array_equal(a, b)


def test_screen_equals_plain_medium(T):
    w = synth.box_precision(seed=5, n=150000, side=500.0)
    res = []
    for precision in (SCREEN, PLAIN):
        with T.Context(precision=precision) as ctx:
            res.append(g3(ctx, w.data, w.rand, w.edges))
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)
    n = len(w.data)
    assert int(res[0][0].sum()) == n * (n - 1) // 2


def test_patches_and_jackknife_3d(T):
    sizes = [0, 1, 300, 900, 257, 1200]
    d = synth.box_clustered(sum(sizes), 12, 1.5, 80.0, 6)
    r = synth.box_points(2 * sum(sizes), 80.0, 7)
    doff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    roff = 2 * doff
    edges = synth.log_edges_r(0.5, 20.0, 10)
    with T.Context() as ctx:
        cd, cr, b = ctx.catalog3d(d, offsets=doff), ctx.catalog3d(r, offsets=roff), ctx.bins3d(edges)
        h = ctx.count_patches(cd, cr, b)
        loo, w, cov = ctx.jackknife(cd, cr, b)
    for p in range(len(sizes)):
        dp, rp = d[doff[p]:doff[p + 1]], r[roff[p]:roff[p + 1]]
        for k, want in enumerate(o3(dp, rp, edges)):
            np.testing.assert_array_equal(h[p, k], want)
    want_loo, want_w, want_cov = oracle.jackknife(d, r, doff, roff, edges, threads=THREADS, euclid=True)
    np.testing.assert_array_equal(loo, want_loo)
    np.testing.assert_array_equal(w, want_w)
    np.testing.assert_array_equal(cov, want_cov)


def test_mixing_angular_and_3d_is_refused(T):
    unit = synth.randoms(100, synth.Footprint("octant"), 1)
    with T.Context() as ctx:
        c_unit, c_3d = ctx.catalog(unit), ctx.catalog3d(unit * 5.0)
        with pytest.raises(T.TpcfError):
            ctx.count_auto(c_unit, ctx.bins3d(np.array([0.0, 1.0])))
        with pytest.raises(T.TpcfError):
            ctx.count_auto(c_3d, ctx.bins(synth.linear_edges(0.0, 5.0, 4)))
        with pytest.raises(T.TpcfError):
            ctx.catalog3d(np.array([[np.nan, 0.0, 0.0]]))
        with pytest.raises(T.TpcfError):
            ctx.catalog3d(np.array([[1e29, 0.0, 0.0]]))
        with pytest.raises(T.TpcfError):
            ctx.bins3d(np.array([0.0, 1e19]))


@pytest.mark.parametrize("precision", [SCREEN, PLAIN])
def test_coordinates_near_the_limit(T, precision):
    # coordinates near 1e27: the FP32 screen bounds overflow, so every pair takes
    # the binary64 recheck, padding pairs (NaN apart) included
    rng = np.random.default_rng(12)
    d = rng.uniform(-1e27, 1e27, (1500, 3))
    r = np.concatenate([d[:300] + rng.normal(0, 3e17, (300, 3)), rng.uniform(-1e27, 1e27, (900, 3))])
    edges = np.array([0.0, 1e16, 1e17, 3e17, 1e18])
    with T.Context(precision=precision) as ctx:
        got, st = ctx.count_all(ctx.catalog3d(d), ctx.catalog3d(r), ctx.bins3d(edges), stats=True)
    assert st["device_error"] == 0
    for a, b in zip(got, o3(d, r, edges)):
        np.testing.assert_array_equal(a, b)
