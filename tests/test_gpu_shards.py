"""The counting kernel on shards of the pair space (tpcf_config.shard_index /
shard_count, one process per GPU in production; here every shard runs in
turn on one GPU): the shards' histograms sum to the unsplit ones, which equal
the oracle's; with more items than blocks, so the dynamic item draws of every
shard's launch are exercised."""
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


def _count(T, d, r, edges, **kw):
    with T.Context(**kw) as ctx:
        (dd, dr, rr), st = ctx.count_all(ctx.catalog(d), ctx.catalog(r), ctx.bins(edges), stats=True)
    assert st["device_error"] == 0
    return np.stack([dd, dr, rr]), st["pairs"]


@pytest.mark.parametrize("world", [2, 3, 5])
def test_shards_sum_to_the_unsplit_histograms(T, world):
    d = synth.clustered(60000, 256, 0.3, seed=21)
    r = synth.randoms(90000, seed=22)
    edges = synth.log_edges(0.02, 6.0, 30)
    full, pairs = _count(T, d, r, edges, threads=128, ipt=8)
    parts = [_count(T, d, r, edges, threads=128, ipt=8, shard_index=s, shard_count=world) for s in range(world)]
    np.testing.assert_array_equal(np.sum([p[0] for p in parts], axis=0, dtype=np.uint64), full)
    assert sum(p[1] for p in parts) == pairs


def test_shards_against_the_oracle(T):
    w = synth.octant_small(seed=5, n=6000)
    want = np.stack([oracle.count_auto(w.data, w.edges, THREADS), oracle.count_cross(w.data, w.rand, w.edges, THREADS),
                     oracle.count_auto(w.rand, w.edges, THREADS)])
    parts = [_count(T, w.data, w.rand, w.edges, threads=128, ipt=8, shard_index=s, shard_count=3)[0] for s in range(3)]
    np.testing.assert_array_equal(np.sum(parts, axis=0, dtype=np.uint64), want)
