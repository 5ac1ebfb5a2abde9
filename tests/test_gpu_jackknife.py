"""Leave-one-out jackknife on the GPU (tpcf_jackknife) against the oracle's
recount of every resampling, and against independent GPU recounts."""
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


def patches(sizes_d, sizes_r, seed):
    fp = synth.Footprint("octant")
    d = synth._band_sort(synth.clustered(int(sum(sizes_d)), 16, 0.3, fp, seed))
    r = synth._band_sort(synth.randoms(int(sum(sizes_r)), fp, seed + 1))
    return d, r, np.concatenate([[0], np.cumsum(sizes_d)]).astype(np.uint64), \
        np.concatenate([[0], np.cumsum(sizes_r)]).astype(np.uint64)


@pytest.mark.parametrize("estimator", [0, 1])
def test_jackknife_equals_oracle(T, estimator):
    sizes_d = [0, 1, 37, 500, 1200, 800, 257]
    sizes_r = [3, 0, 90, 1000, 700, 1500, 255]
    d, r, doff, roff = patches(sizes_d, sizes_r, seed=11)
    edges = synth.linear_edges(0.0, 6.0, 24)
    with T.Context() as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        loo, w, cov, st = ctx.jackknife(cd, cr, b, estimator=estimator, stats=True)
    assert st["device_error"] == 0
    want_loo, want_w, want_cov = oracle.jackknife(d, r, doff, roff, edges, estimator, THREADS)
    np.testing.assert_array_equal(loo, want_loo)
    np.testing.assert_array_equal(w, want_w)
    np.testing.assert_array_equal(cov, want_cov)


def test_jackknife_equals_gpu_recounts(T):
    rng = np.random.default_rng(4)
    sizes_d = rng.integers(500, 6000, 20)
    sizes_r = 2 * sizes_d
    d, r, doff, roff = patches(sizes_d, sizes_r, seed=12)
    edges = synth.log_edges(0.02, 5.0, 30)
    with T.Context() as ctx:
        cd, cr, b = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff), ctx.bins(edges)
        loo, w, cov = ctx.jackknife(cd, cr, b)
        full = ctx.count_all(ctx.catalog(d), ctx.catalog(r), b)
        for p in (0, 7, 19):
            dp = np.concatenate([d[:doff[p]], d[doff[p + 1]:]])
            rp = np.concatenate([r[:roff[p]], r[roff[p + 1]:]])
            got = ctx.count_all(ctx.catalog(dp), ctx.catalog(rp), b)
            for k in range(3):
                np.testing.assert_array_equal(loo[p, k], got[k], err_msg=f"patch {p} kind {k}")
    # every resampling drops pairs, none adds any
    for k in range(3):
        assert np.all(loo[:, k].astype(np.int64) <= full[k].astype(np.int64))
    assert np.all(np.linalg.eigvalsh(cov) > -1e-12 * np.abs(cov).max())


def test_jackknife_rejects_bad_input(T):
    d, r, doff, roff = patches([100, 200], [150, 250], seed=13)
    with T.Context() as ctx:
        cd, cr = ctx.catalog(d, offsets=doff), ctx.catalog(r, offsets=roff)
        with pytest.raises(T.TpcfError):  # range past 90 degrees
            ctx.jackknife(cd, cr, ctx.bins(synth.linear_edges(0.0, 120.0, 10)))
        with pytest.raises(T.TpcfError):  # random catalog not segmented
            ctx.jackknife(cd, ctx.catalog(r), ctx.bins(synth.linear_edges(0.0, 5.0, 10)))
