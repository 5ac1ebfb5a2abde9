"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Histograms must be identical integer for integer; w(theta) agrees to a
relative 1e-12 (both sides evaluate the same binary64 formula).  Sizes span
several tiles and ragged tails; edge cases cover empty and tiny catalogs,
duplicates, antipodes, edges at 0 and pi, bins inside the FP32 guard band and
one-bin / many-bin sets.
"""
import math
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


@pytest.fixture(scope="module")
def ctxs(T):
    c = {SCREEN: T.Context(precision=SCREEN), PLAIN: T.Context(precision=PLAIN)}
    yield c
    for v in c.values():
        v.close()


def gpu_auto(ctx, x, edges, **kw):
    cat = ctx.catalog(x)
    b = ctx.bins(edges)
    try:
        return ctx.count_auto(cat, b, **kw)
    finally:
        ctx.free(cat)
        ctx.free(b)


def gpu_cross(ctx, x, y, edges, **kw):
    a = ctx.catalog(x)
    c = ctx.catalog(y)
    b = ctx.bins(edges)
    try:
        return ctx.count_cross(a, c, b, **kw)
    finally:
        for o in (a, c, b):
            ctx.free(o)


# ------------------------------------------------------------------ golden fixtures
@pytest.mark.parametrize("prec", [SCREEN, PLAIN])
def test_golden_fixtures(ctxs, prec):
    from tests.golden import FIXTURES, load_fixture
    for name in FIXTURES:
        fx = load_fixture(name)
        if fx["kind"] == "auto":
            got = gpu_auto(ctxs[prec], fx["a"], fx["edges"])
        else:
            got = gpu_cross(ctxs[prec], fx["a"], fx["b"], fx["edges"])
        np.testing.assert_array_equal(got, fx["hist"], err_msg=name)


# ------------------------------------------------------------------ the small octant workload
@pytest.fixture(scope="module")
def small():
    w = synth.octant_small(seed=0)
    return w, oracle.correlation(w.data, w.rand, w.edges, threads=THREADS)


@pytest.mark.parametrize("prec", [SCREEN, PLAIN])
def test_octant_small_full_exact(ctxs, small, prec):
    w, (odd, odr, orr, ow) = small
    ctx = ctxs[prec]
    d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
    (dd, dr, rr), st = ctx.count_all(d, r, b, stats=True)
    np.testing.assert_array_equal(dd, odd)
    np.testing.assert_array_equal(dr, odr)
    np.testing.assert_array_equal(rr, orr)
    assert st["pairs"] == w.pairs and st["device_error"] == 0
    # separate launches give the same histograms
    np.testing.assert_array_equal(ctx.count_auto(d, b), odd)
    np.testing.assert_array_equal(ctx.count_auto(r, b), orr)
    np.testing.assert_array_equal(ctx.count_cross(d, r, b), odr)
    for o in (d, r, b):
        ctx.free(o)


def test_octant_small_w_matches_oracle(ctxs, small):
    w, (odd, odr, orr, ow) = small
    for est in (0, 1):
        dd, dr, rr, wt = ctxs[SCREEN].correlate(w.data, w.rand, w.edges, estimator=est)
        np.testing.assert_array_equal(dd, odd)
        ow_e = oracle.estimate(odd[1:-1], odr[1:-1], orr[1:-1], len(w.data), len(w.rand), est)
        np.testing.assert_allclose(wt, ow_e, rtol=1e-12, atol=0)


# ------------------------------------------------------------------ ragged sizes and shapes
# (j-tiles of each warp's ring: every shape fits both the FP32 and the binary64 staging)
SHAPES = [dict(threads=128, ipt=8, jtile=512), dict(threads=256, ipt=8, jtile=256),
          dict(threads=512, ipt=8, jtile=128), dict(threads=256, ipt=16, jtile=256)]


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("prec", [SCREEN, PLAIN])
def test_ragged_sizes_and_shapes(T, shape, prec):
    edges = synth.log_edges(0.01, 10.0, 64)
    with T.Context(precision=prec, **SHAPES[shape]) as ctx:
        for n in (1, 2, 3, 33, 1000, 4095, 4097, 6001):
            x = synth.clustered(n, 16, 0.2, synth.Footprint("octant"), seed=n)
            y = synth.randoms(n + 77, seed=n)
            np.testing.assert_array_equal(gpu_auto(ctx, x, edges), oracle.count_auto(x, edges, THREADS),
                                          err_msg=f"auto n={n}")
            np.testing.assert_array_equal(gpu_cross(ctx, x, y, edges),
                                          oracle.count_cross(x, y, edges, THREADS), err_msg=f"cross n={n}")


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("prec", [SCREEN, PLAIN])
def test_one_bin_holding_every_pair_at_every_shape(T, shape, prec):
    # edges [0, pi]: every pair lands in one bin, so one lane's 16-bit counter of that row takes
    # R x J increments per tile (16 x 4096 per item at 256 x 16); the warp must merge it before
    # it passes 2^16 - 1, or it would carry into its partner's half of the shared word
    edges = np.array([0.0, math.pi])
    n = 20_000
    x = synth.clustered(n, 16, 0.2, synth.Footprint("octant"), seed=11)
    y = synth.randoms(n + 999, seed=12)
    with T.Context(precision=prec, **SHAPES[shape]) as ctx:
        auto, cross = gpu_auto(ctx, x, edges), gpu_cross(ctx, x, y, edges)
    np.testing.assert_array_equal(auto, [0, n * (n - 1) // 2, 0])
    np.testing.assert_array_equal(cross, [0, n * (n + 999), 0])
    np.testing.assert_array_equal(auto, oracle.count_auto(x, edges, THREADS))
    np.testing.assert_array_equal(cross, oracle.count_cross(x, y, edges, THREADS))


def test_empty_catalogs(ctxs):
    edges = synth.linear_edges(0.0, 10.0, 40)
    z = np.zeros((0, 3))
    x = synth.randoms(100, seed=1)
    for prec in (SCREEN, PLAIN):
        assert not gpu_auto(ctxs[prec], z, edges).any()
        assert not gpu_cross(ctxs[prec], z, x, edges).any()
        assert not gpu_cross(ctxs[prec], x, z, edges).any()


# ------------------------------------------------------------------ edge sets
EDGE_SETS = {
    "one_bin": np.array([0.1, 5.0]) * math.pi / 180,
    "many_bins": synth.linear_edges(0.0, 20.0, 128),
    "to_pi": np.linspace(0.0, math.pi, 13),
    "tiny_angles": synth.log_edges(0.0005, 0.05, 24),
    "wide_log": synth.log_edges(0.001, 179.0, 300),
}


@pytest.mark.parametrize("name", sorted(EDGE_SETS))
@pytest.mark.parametrize("prec", [SCREEN, PLAIN])
def test_edge_sets(ctxs, name, prec):
    edges = EDGE_SETS[name]
    x = synth.clustered(3000, 8, 0.05, synth.Footprint("sphere"), seed=3)
    y = synth.randoms(2500, synth.Footprint("sphere"), seed=4)
    np.testing.assert_array_equal(gpu_auto(ctxs[prec], x, edges), oracle.count_auto(x, edges, THREADS))
    np.testing.assert_array_equal(gpu_cross(ctxs[prec], x, y, edges),
                                  oracle.count_cross(x, y, edges, THREADS))


def test_duplicates_antipodes_and_identical_points(ctxs):
    base = synth.randoms(700, synth.Footprint("sphere"), seed=8)
    x = np.concatenate([base, base, -base[:200], np.repeat(base[:1], 300, axis=0)])
    for edges in (synth.linear_edges(0.0, 180.0, 36), synth.log_edges(1e-4, 1.0, 30),
                  np.array([1e-7, 1e-3, math.pi])):
        want = oracle.count_auto(x, edges, THREADS)
        for prec in (SCREEN, PLAIN):
            np.testing.assert_array_equal(gpu_auto(ctxs[prec], x, edges), want)


def test_pairs_straddling_every_edge(ctxs):
    # For each edge t_k, point pairs at t_k (1 +/- eps) for eps from 1e-9 to 1e-3,
    # placed along random great circles: these pairs sit inside the FP32 guard
    # band and exercise the binary64 recheck.
    rng = np.random.default_rng(12)
    edges = synth.log_edges(0.01, 10.0, 64)
    a, b = [], []
    for t in edges:
        for eps in (-1e-3, -1e-5, -1e-7, -1e-9, 1e-9, 1e-7, 1e-5, 1e-3):
            u = rng.normal(size=3); u /= np.linalg.norm(u)
            v = rng.normal(size=3); v -= (v @ u) * u; v /= np.linalg.norm(v)
            s = t * (1 + eps)
            a.append(u)
            q = math.cos(s) * u + math.sin(s) * v
            b.append(q / np.linalg.norm(q))
    a, b = np.array(a), np.array(b)
    want = oracle.count_cross(a, b, edges)
    for prec in (SCREEN, PLAIN):
        got, st = ctxs[prec].count_cross(ctxs[prec].catalog(a), ctxs[prec].catalog(b),
                                         ctxs[prec].bins(edges), stats=True)
        np.testing.assert_array_equal(got, want)
        if prec == SCREEN:
            assert st["band_pairs"] > 0


# ------------------------------------------------------------------ screen vs plain at size
def test_screen_equals_plain_200k(ctxs):
    w = synth.octant_precision(seed=1, n=200_000)
    res = {}
    for prec in (SCREEN, PLAIN):
        ctx = ctxs[prec]
        d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
        res[prec] = ctx.count_all(d, r, b, stats=True)
        for o in (d, r, b):
            ctx.free(o)
    (s_h, s_st), (p_h, p_st) = res[SCREEN], res[PLAIN]
    for a, c in zip(s_h, p_h):
        np.testing.assert_array_equal(a, c)
    assert s_st["pairs"] == p_st["pairs"] == w.pairs
    assert s_st["band_pairs"] > 0
    n = 200_000
    assert int(s_h[0].sum()) == n * (n - 1) // 2 and int(s_h[1].sum()) == n * n


def test_sort_does_not_change_counts(T, ctxs):
    w = synth.octant_small(seed=2, n=5000)
    with T.Context(flags=T.TPCF_F_NO_SORT) as raw:
        d, r, b = raw.catalog(w.data), raw.catalog(w.rand), raw.bins(w.edges)
        unsorted = raw.count_all(d, r, b)
    ctx = ctxs[SCREEN]
    d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
    for a, c in zip(unsorted, ctx.count_all(d, r, b)):
        np.testing.assert_array_equal(a, c)
    for o in (d, r, b):
        ctx.free(o)


# ------------------------------------------------------------------ device buffers and streams
def test_device_inputs_outputs_and_concurrent_streams(ctxs):
    import torch
    w = synth.octant_small(seed=3, n=6000)
    ctx = ctxs[SCREEN]
    dd_ref, dr_ref, rr_ref = (ctx.count_all(ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)))
    dev_d = torch.from_numpy(w.data).cuda()
    dev_r = torch.from_numpy(w.rand).cuda()
    d, r, b = ctx.catalog(dev_d), ctx.catalog(dev_r), ctx.bins(w.edges)
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs = [torch.zeros(len(w.edges) + 1, dtype=torch.int64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    ctx.count_auto(d, b, stream=streams[0], out=outs[0])
    ctx.count_cross(d, r, b, stream=streams[1], out=outs[1])
    ctx.count_auto(r, b, stream=streams[2], out=outs[2])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(outs[0].cpu().numpy().view(np.uint64), dd_ref)
    np.testing.assert_array_equal(outs[1].cpu().numpy().view(np.uint64), dr_ref)
    np.testing.assert_array_equal(outs[2].cpu().numpy().view(np.uint64), rr_ref)


# ------------------------------------------------------------------ errors
def test_invalid_points_rejected(T, ctxs):
    ctx = ctxs[SCREEN]
    x = synth.randoms(100, seed=5)
    bad = x.copy(); bad[17, 0] = np.nan
    with pytest.raises(T.TpcfError) as ei:
        ctx.catalog(bad)
    assert ei.value.status == T.TPCF_EINVAL
    bad = x.copy(); bad[3] *= 1.01
    with pytest.raises(T.TpcfError):
        ctx.catalog(bad)
    with pytest.raises(T.TpcfError):
        ctx.bins(np.array([0.3, 0.2]))


def test_bounded_wait_timeout_reports_and_context_survives(T, ctxs):
    # The test hook leaves the first j-tile copy unissued: every block's wait on
    # it runs out after 20 ms, the kernel sets its error word and returns.
    x = synth.randoms(3000, seed=6)
    edges = synth.linear_edges(0.0, 10.0, 10)
    with T.Context(flags=T.TPCF_F_TEST_WAIT_TIMEOUT, wait_timeout_us=20000) as bad:
        with pytest.raises(T.TpcfError) as ei:
            gpu_auto(bad, x, edges)
        assert ei.value.status == T.TPCF_ETIMEOUT
        # the same context keeps working for a call that does not wait
        assert not gpu_auto(bad, np.zeros((0, 3)), edges).any()
    np.testing.assert_array_equal(gpu_auto(ctxs[SCREEN], x, edges), oracle.count_auto(x, edges, THREADS))


def test_allocation_failure_reported(T, ctxs):
    x = synth.randoms(1000, seed=7)
    T.tpcf_debug_fail_alloc_after(0)
    try:
        with pytest.raises(T.TpcfError) as ei:
            ctxs[SCREEN].catalog(x)
        assert ei.value.status == T.TPCF_ENOMEM
    finally:
        T.tpcf_debug_fail_alloc_after(-1)
    assert ctxs[SCREEN].catalog(x).n == 1000
