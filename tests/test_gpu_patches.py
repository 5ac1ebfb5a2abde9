"""Jackknife patches: per-patch DD, DR, RR of segmented catalogs in one launch.

The batched launch must give, for every patch, exactly the histograms of the
oracle on that patch alone, and of separate library launches on the patch's
points; empty and one-point patches included.
"""
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


def patch_set(sizes_d, seed=0):
    """Band-sorted octant catalogs cut into consecutive patches."""
    nd = int(sum(sizes_d))
    d = synth._band_sort(synth.clustered(nd, 16, 0.3, synth.Footprint("octant"), seed))
    r = synth._band_sort(synth.randoms(2 * nd, synth.Footprint("octant"), seed))
    doff = np.concatenate([[0], np.cumsum(sizes_d)]).astype(np.uint64)
    roff = 2 * doff
    return d, r, doff, roff


def oracle_patch(d, r, doff, roff, p, edges):
    dp = d[int(doff[p]):int(doff[p + 1])]
    rp = r[int(roff[p]):int(roff[p + 1])]
    return (oracle.count_auto(dp, edges, THREADS), oracle.count_cross(dp, rp, edges, THREADS),
            oracle.count_auto(rp, edges, THREADS))


@pytest.mark.parametrize("flags", [0, 0x8])
def test_patches_equal_oracle_per_patch(T, flags):
    sizes = [0, 1, 2, 37, 1000, 4095, 4097, 250, 3000, 1, 0, 777]
    d, r, doff, roff = patch_set(sizes, seed=3)
    edges = synth.linear_edges(0.0, 5.0, 40)
    with T.Context(flags=flags) as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        h, st = ctx.count_patches(cd, cr, b, stats=True)
        assert st["device_error"] == 0
        for p in range(len(sizes)):
            want = oracle_patch(d, r, doff, roff, p, edges)
            for k in range(3):
                np.testing.assert_array_equal(h[p, k], want[k], err_msg=f"patch {p} kind {k}")
        want_pairs = sum(n * (n - 1) // 2 + (2 * n) * (2 * n - 1) // 2 + n * 2 * n for n in sizes)
        assert st["pairs"] == want_pairs


def test_patches_equal_separate_launches_and_device_output(T):
    import torch
    rng = np.random.default_rng(5)
    sizes = list(rng.integers(100, 6000, 24))
    d, r, doff, roff = patch_set(sizes, seed=4)
    edges = synth.log_edges(0.01, 5.0, 40)
    with T.Context() as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        h = ctx.count_patches(cd, cr, b)
        hd = ctx.count_patches(cd, cr, b, device_out=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hd.cpu().numpy().view(np.uint64), h)
        for p in range(len(sizes)):
            dp = d[int(doff[p]):int(doff[p + 1])]
            rp = r[int(roff[p]):int(roff[p + 1])]
            a, c = ctx.catalog(dp), ctx.catalog(rp)
            np.testing.assert_array_equal(h[p, 0], ctx.count_auto(a, b))
            np.testing.assert_array_equal(h[p, 1], ctx.count_cross(a, c, b))
            np.testing.assert_array_equal(h[p, 2], ctx.count_auto(c, b))
            ctx.free(a)
            ctx.free(c)


def test_patches_reject_mismatched_segments(T):
    d, r, doff, roff = patch_set([100, 200], seed=6)
    with T.Context() as ctx:
        cd = ctx.catalog(d, offsets=doff)
        cr = ctx.catalog(r)  # not segmented
        with pytest.raises(T.TpcfError):
            ctx.count_patches(cd, cr, ctx.bins(synth.linear_edges(0.0, 5.0, 10)))


@pytest.mark.parametrize("flags", [0, 0x8])
def test_patch_graph_replays_equal_direct_call(T, flags):
    import torch
    rng = np.random.default_rng(9)
    sizes = [0, 1] + list(rng.integers(200, 9000, 30))
    d, r, doff, roff = patch_set(sizes, seed=9)
    edges = synth.linear_edges(0.0, 5.0, 40)
    with T.Context(flags=flags) as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        want = ctx.count_patches(cd, cr, b)
        g = ctx.graph(T.TPCF_GRAPH_PATCHES, cd, cr, b)
        s = torch.cuda.current_stream()
        for _ in range(3):  # each replay clears and recounts
            g.launch(s)
        st = g.stats()
        np.testing.assert_array_equal(g.out.cpu().numpy().view(np.uint64), want)
        assert st["device_error"] == 0 and st["launches"] == 2
        want_pairs = sum(n * (n - 1) // 2 + (2 * n) * (2 * n - 1) // 2 + 2 * n * n for n in sizes)
        assert st["pairs"] == want_pairs


def test_graph_kinds_equal_direct_calls(T):
    import torch
    d = synth.clustered(30000, 64, 0.3, synth.Footprint("octant"), 21)
    r = synth.randoms(45000, synth.Footprint("octant"), 22)
    edges = synth.log_edges(0.01, 10.0, 64)
    with T.Context() as ctx:
        cd, cr, b = ctx.catalog(d), ctx.catalog(r), ctx.bins(edges)
        dd, dr, rr = ctx.count_all(cd, cr, b)
        s = torch.cuda.current_stream()
        ga = ctx.graph(T.TPCF_GRAPH_AUTO, cd, None, b)
        gc = ctx.graph(T.TPCF_GRAPH_CROSS, cd, cr, b)
        gall = ctx.graph(T.TPCF_GRAPH_ALL, cd, cr, b)
        for g in (ga, gc, gall):
            g.launch(s)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ga.out.cpu().numpy().view(np.uint64), dd)
        np.testing.assert_array_equal(gc.out.cpu().numpy().view(np.uint64), dr)
        np.testing.assert_array_equal(gall.out.cpu().numpy().view(np.uint64), np.stack([dd, dr, rr]))
        assert gall.stats()["pairs"] == int(dd.sum() + dr.sum() + rr.sum())
        ctx.free(ga)
        with pytest.raises(T.TpcfError) as e:
            ctx.graph(T.TPCF_GRAPH_PATCHES, cd, cr, b)  # not segmented
        assert e.value.status == T.TPCF_EINVAL
        g_new = ctx.graph(T.TPCF_GRAPH_AUTO, cr, None, b)
        with pytest.raises(T.TpcfError) as e:
            g_new.stats()  # never launched
        assert e.value.status == T.TPCF_ESTATE
