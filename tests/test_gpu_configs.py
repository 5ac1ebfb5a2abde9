"""Parity at the full sizes of the benchmark workloads, in the launch
configurations bench.py times.

The histograms of a full-size problem are single aggregates, so the oracle
cannot check them element by element; parity is shown through properties that
hold at any size (pair totals, identity with the independent all-binary64
kernel, batched == separate launches) and through the oracle on subsamples
and on the smallest units of a workload:
  - 1,000,000 + 1,000,000 octant points, 64 log bins 0.01-10 deg;
  - 2,000,000 + 4,000,000 points in 512 jackknife patches, 40 linear bins 0-5 deg;
  - the 20 smallest jobs of the 2,000-job serving stream, through the job server;
  - 4,000,000 + 8,000,000 full-sphere points, 80 log bins 0.005-2 deg.
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


def oracle_all(d, r, edges):
    return (oracle.count_auto(d, edges, THREADS), oracle.count_cross(d, r, edges, THREADS),
            oracle.count_auto(r, edges, THREADS))


def totals_hold(dd, dr, rr, nd, nr):
    return (int(dd.sum()) == nd * (nd - 1) // 2 and int(dr.sum()) == nd * nr
            and int(rr.sum()) == nr * (nr - 1) // 2)


def test_octant_precision_full_size(T):
    import torch
    w = synth.octant_precision(seed=0)
    dev_d, dev_r = torch.from_numpy(w.data).cuda(), torch.from_numpy(w.rand).cuda()
    with T.Context() as ctx:
        cd, cr, b = ctx.catalog(dev_d), ctx.catalog(dev_r), ctx.bins(w.edges)
        (dd, dr, rr), st = ctx.count_all(cd, cr, b, stats=True)
        # the same catalogs, reordered: counts do not depend on the order
        perm = np.random.default_rng(1).permutation(len(w.data))
        cdp = ctx.catalog(w.data[perm])
        np.testing.assert_array_equal(ctx.count_auto(cdp, b), dd)
    assert st["device_error"] == 0 and st["launches"] >= 1
    assert totals_hold(dd, dr, rr, len(w.data), len(w.rand))
    with T.Context(precision=T.TPCF_PLAIN_FP64) as ctx:
        cd, cr, b = ctx.catalog(dev_d), ctx.catalog(dev_r), ctx.bins(w.edges)
        pdd, pdr, prr = ctx.count_all(cd, cr, b)
    for got, want in zip((dd, dr, rr), (pdd, pdr, prr)):
        np.testing.assert_array_equal(got, want)
    # a random subsample of each catalog against the oracle
    g = np.random.default_rng(2)
    ds = w.data[np.sort(g.choice(len(w.data), 20000, replace=False))]
    rs = w.rand[np.sort(g.choice(len(w.rand), 20000, replace=False))]
    with T.Context() as ctx:
        got = ctx.count_all(ctx.catalog(ds), ctx.catalog(rs), ctx.bins(w.edges))
    for g_, o_ in zip(got, oracle_all(ds, rs, w.edges)):
        np.testing.assert_array_equal(g_, o_)


def test_jackknife_full_size(T):
    d, r, doff, roff = synth.jackknife_patches(seed=0)
    edges = synth.linear_edges(0.0, 5.0, 40)
    nd_p = np.diff(doff)
    with T.Context(flags=T.TPCF_F_AUTOTUNE) as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        g = ctx.graph(T.TPCF_GRAPH_PATCHES, cd, cr, b)
        g.launch()
        st = g.stats()
        h = g.out.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(ctx.count_patches(cd, cr, b), h)
        want_pairs = sum(n * (n - 1) // 2 + (2 * n) * (2 * n - 1) // 2 + 2 * n * n for n in nd_p.tolist())
        assert st["pairs"] == want_pairs and st["device_error"] == 0
        # separate launches on a sample of patches
        for p in np.random.default_rng(3).choice(len(nd_p), 24, replace=False):
            dp, rp = d[doff[p]:doff[p + 1]], r[roff[p]:roff[p + 1]]
            a, c = ctx.catalog(dp), ctx.catalog(rp)
            np.testing.assert_array_equal(h[p, 0], ctx.count_auto(a, b))
            np.testing.assert_array_equal(h[p, 1], ctx.count_cross(a, c, b))
            np.testing.assert_array_equal(h[p, 2], ctx.count_auto(c, b))
            ctx.free(a)
            ctx.free(c)
    # the oracle on the 16 smallest patches and the largest one
    order = np.argsort(nd_p, kind="stable")
    for p in list(order[:16]) + [order[-1]]:
        dp, rp = d[doff[p]:doff[p + 1]], r[roff[p]:roff[p + 1]]
        for k, want in enumerate(oracle_all(dp, rp, edges)):
            np.testing.assert_array_equal(h[p, k], want, err_msg=f"patch {p} kind {k}")


def test_serving_smallest_jobs_through_the_server(T):
    specs = synth.serving_jobs(2000, seed=0)
    smallest = sorted(specs, key=lambda s: s["nd"])[:20]
    jobs = [synth.materialise_job(s) for s in smallest]
    with T.Context(server_workers=4, hbm_budget_bytes=120 << 30) as ctx:
        ids = [ctx.submit(w.data, w.rand, w.edges) for w in jobs]
        for jid, w in zip(ids, jobs):
            res = ctx.poll(jid, len(w.edges))
            dd, dr, rr = oracle_all(w.data, w.rand, w.edges)
            np.testing.assert_array_equal(res["dd"], dd)
            np.testing.assert_array_equal(res["dr"], dr)
            np.testing.assert_array_equal(res["rr"], rr)
            want_w = oracle.estimate(dd[1:-1], dr[1:-1], rr[1:-1], len(w.data), len(w.rand))
            np.testing.assert_array_equal(res["w"], want_w)


def test_sphere_large_full_size(T):
    import torch
    w = synth.sphere_large(seed=0)
    nd, nr = len(w.data), len(w.rand)
    with T.Context() as ctx:
        cd = ctx.catalog(torch.from_numpy(w.data).cuda())
        cr = ctx.catalog(torch.from_numpy(w.rand).cuda())
        b = ctx.bins(w.edges)
        (dd, dr, rr), st = ctx.count_all(cd, cr, b, stats=True)
        assert st["device_error"] == 0 and st["pairs"] == nd * (nd - 1) // 2 + nd * nr + nr * (nr - 1) // 2
        assert totals_hold(dd, dr, rr, nd, nr)
        g = np.random.default_rng(7)
        ds = w.data[np.sort(g.choice(nd, 30000, replace=False))]
        rs = w.rand[np.sort(g.choice(nr, 30000, replace=False))]
        got = ctx.count_all(ctx.catalog(ds), ctx.catalog(rs), b)
    for g_, o_ in zip(got, oracle_all(ds, rs, w.edges)):
        np.testing.assert_array_equal(g_, o_)


def test_jackknife_leave_one_out_full_size(T):
    d, r, doff, roff = synth.jackknife_patches(seed=0)
    edges = synth.linear_edges(0.0, 5.0, 40)
    with T.Context() as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        loo, w, cov, st = ctx.jackknife(cd, cr, b, stats=True)
        assert st["device_error"] == 0
        nd, nr = len(d), len(r)
        for p in range(len(doff) - 1):
            a, c = nd - int(doff[p + 1] - doff[p]), nr - int(roff[p + 1] - roff[p])
            assert int(loo[p, 0].sum()) == a * (a - 1) // 2 and int(loo[p, 1].sum()) == a * c
            assert int(loo[p, 2].sum()) == c * (c - 1) // 2
        for p in (0, 311):  # two resamplings recounted from scratch
            dp = np.concatenate([d[:doff[p]], d[doff[p + 1]:]])
            rp = np.concatenate([r[:roff[p]], r[roff[p + 1]:]])
            got = ctx.count_all(ctx.catalog(dp), ctx.catalog(rp), b)
            for k in range(3):
                np.testing.assert_array_equal(loo[p, k], got[k], err_msg=f"patch {p} kind {k}")
    assert np.all(np.isfinite(np.diag(cov)))
