"""The overflow checksum mode (TPCF_F_CHECK_OVERFLOW) through the C ABI.

Normally the finalize derives each histogram's overflow entry as the pair total
minus the other entries, so a pair the kernel lost would hide there.  With the
flag the kernels count the overflow row like every other row (the pairs the
FP32 screen rejects included) and the call fails when a histogram does not sum
to its pair total.  Here: the counted overflow equals the oracle's on the
small octant workload (both precisions, fused and separate launches), on
ragged sizes across the kernel shapes, on patches and in 3-D; the 200k + 200k
screen equals the all-binary64 kernel with counted overflow; at 1M + 1M (every
phase of the launch's draw order) and through the job server's steps the
checked calls succeed with the usual histograms; and a test hook that checks
against the pair total plus one makes the call fail while the context stays
usable.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import build, synth

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
SCREEN, PLAIN = 0, 1
SHAPES = [dict(threads=128, ipt=8, jtile=512), dict(threads=256, ipt=8, jtile=256),
          dict(threads=512, ipt=8, jtile=128), dict(threads=256, ipt=16, jtile=256)]


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1204_6630_gb300 import tpcf
    tpcf.load()
    return tpcf


@pytest.fixture(scope="module")
def small():
    w = synth.octant_small(seed=0)
    return w, oracle.correlation(w.data, w.rand, w.edges, threads=THREADS)


@pytest.mark.parametrize("prec", [SCREEN, PLAIN])
def test_counted_overflow_equals_the_oracle_on_the_small_octant(T, small, prec):
    w, (odd, odr, orr, _) = small
    with T.Context(precision=prec, flags=T.TPCF_F_CHECK_OVERFLOW) as ctx:
        d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
        (dd, dr, rr), st = ctx.count_all(d, r, b, stats=True)
        for got, want in zip((dd, dr, rr), (odd, odr, orr)):
            np.testing.assert_array_equal(got, want)
        assert st["device_error"] == 0 and st["pairs"] == w.pairs
        np.testing.assert_array_equal(ctx.count_auto(d, b), odd)
        np.testing.assert_array_equal(ctx.count_auto(r, b), orr)
        np.testing.assert_array_equal(ctx.count_cross(d, r, b), odr)


def test_screen_equals_plain_with_counted_overflow_at_200k(T):
    w = synth.octant_precision(seed=1, n=200_000)
    res = {}
    for prec in (SCREEN, PLAIN):
        with T.Context(precision=prec, flags=T.TPCF_F_CHECK_OVERFLOW) as ctx:
            d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
            res[prec] = ctx.count_all(d, r, b, stats=True)
    with T.Context() as ctx:  # the derived overflow, for comparison
        d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
        derived = ctx.count_all(d, r, b)
    (s_h, s_st), (p_h, p_st) = res[SCREEN], res[PLAIN]
    for a, c, e in zip(s_h, p_h, derived):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(a, e)
    assert s_st["device_error"] == 0 and p_st["device_error"] == 0
    n = 200_000
    assert int(s_h[0].sum()) == n * (n - 1) // 2 and int(s_h[1].sum()) == n * n


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_counted_overflow_on_ragged_sizes_and_shapes(T, shape):
    # diagonal and padded tiles take every group through the slow path in this mode
    edges = synth.log_edges(0.01, 10.0, 64)
    with T.Context(flags=T.TPCF_F_CHECK_OVERFLOW, **SHAPES[shape]) as ctx:
        for n in (1, 2, 33, 1000, 4097, 6001):
            x = synth.clustered(n, 16, 0.2, synth.Footprint("octant"), seed=n)
            y = synth.randoms(n + 77, seed=n)
            cx, cy, b = ctx.catalog(x), ctx.catalog(y), ctx.bins(edges)
            np.testing.assert_array_equal(ctx.count_auto(cx, b), oracle.count_auto(x, edges, THREADS),
                                          err_msg=f"auto n={n}")
            np.testing.assert_array_equal(ctx.count_cross(cx, cy, b), oracle.count_cross(x, y, edges, THREADS),
                                          err_msg=f"cross n={n}")
            for o in (cx, cy, b):
                ctx.free(o)


def test_counted_overflow_on_patches(T):
    sizes = [0, 1, 37, 1000, 4097, 250, 1]
    nd = int(sum(sizes))
    d = synth._band_sort(synth.clustered(nd, 16, 0.3, synth.Footprint("octant"), 5))
    r = synth._band_sort(synth.randoms(2 * nd, synth.Footprint("octant"), 5))
    doff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    roff = 2 * doff
    edges = synth.linear_edges(0.0, 5.0, 40)
    with T.Context(flags=T.TPCF_F_CHECK_OVERFLOW) as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        h = ctx.count_patches(cd, cr, b)
    for p in range(len(sizes)):
        dp, rp = d[int(doff[p]):int(doff[p + 1])], r[int(roff[p]):int(roff[p + 1])]
        want = (oracle.count_auto(dp, edges, THREADS), oracle.count_cross(dp, rp, edges, THREADS),
                oracle.count_auto(rp, edges, THREADS))
        for k in range(3):
            np.testing.assert_array_equal(h[p, k], want[k], err_msg=f"patch {p} kind {k}")


def test_counted_overflow_in_3d(T):
    edges = synth.log_edges_r(0.5, 50.0, 30)
    d = synth.box_clustered(5000, 40, 2.0, 300.0, 2)
    r = synth.box_points(7000, 300.0, 3)
    with T.Context(flags=T.TPCF_F_CHECK_OVERFLOW) as ctx:
        cd, cr, b = ctx.catalog3d(d), ctx.catalog3d(r), ctx.bins3d(edges)
        dd, dr, rr = ctx.count_all(cd, cr, b)
    np.testing.assert_array_equal(dd, oracle.count_auto(d, edges, THREADS, euclid=True))
    np.testing.assert_array_equal(dr, oracle.count_cross(d, r, edges, THREADS, euclid=True))
    np.testing.assert_array_equal(rr, oracle.count_auto(r, edges, THREADS, euclid=True))


def test_a_histogram_that_does_not_add_up_fails_the_call(T):
    w = synth.octant_small(seed=4, n=3000)
    with T.Context(flags=T.TPCF_F_CHECK_OVERFLOW | T.TPCF_F_TEST_BAD_TOTAL) as bad:
        d, b = bad.catalog(w.data), bad.bins(w.edges)
        with pytest.raises(T.TpcfError) as ei:
            bad.count_auto(d, b)
        assert ei.value.status == T.TPCF_ECUDA
        assert "does not add up" in str(ei.value)
    # the device and a fresh context are still usable, and the check passes without the hook
    with T.Context(flags=T.TPCF_F_CHECK_OVERFLOW) as ctx:
        d, b = ctx.catalog(w.data), ctx.bins(w.edges)
        np.testing.assert_array_equal(ctx.count_auto(d, b), oracle.count_auto(w.data, w.edges, THREADS))


def test_counted_overflow_at_1m_covers_every_draw_phase(T):
    # 1.9e6 items against 64 x 2432 late items: the walk-order middle of the range runs too, so
    # an item the draw order dropped or counted twice would make the checked call fail
    w = synth.octant_precision(seed=0, n=1_000_000)
    with T.Context() as ctx:
        d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
        derived = ctx.count_all(d, r, b)
    with T.Context(flags=T.TPCF_F_CHECK_OVERFLOW) as ctx:
        d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
        counted, st = ctx.count_all(d, r, b, stats=True)
    for a, c in zip(counted, derived):
        np.testing.assert_array_equal(a, c)
    assert st["device_error"] == 0 and st["pairs"] == w.pairs


def test_counted_overflow_through_the_job_server(T):
    # small jobs share the multi-job kernel's steps, the largest runs in preemptible one-job steps
    specs = synth.serving_jobs(24, seed=5)
    jobs = [synth.materialise_job(s) for s in specs]
    with T.Context() as lone:
        want = [lone.correlate(j.data, j.rand, j.edges) for j in jobs]
    with T.Context(flags=T.TPCF_F_CHECK_OVERFLOW) as ctx:
        ids = [ctx.submit(j.data, j.rand, j.edges) for j in jobs]
        got = [ctx.poll(i, len(j.edges)) for i, j in zip(ids, jobs)]
    for g, w_ in zip(got, want):
        for k, name in enumerate(("dd", "dr", "rr")):
            np.testing.assert_array_equal(g[name], w_[k])
