"""Multi-process split of the pair space (host side, gloo, world size 2).

Each rank takes its shard of the counting kernel's work items (the split of
``tpcf_config.shard_index/shard_count``, enumerated by the library's own plan
code), computes the histogram of exactly those pairs with the oracle, and the
ranks sum their histograms with an all-reduce.  The sum must equal the
unsplit oracle histogram and every pair must be covered exactly once.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import build, synth

N, NR = 70, 53
I, JC, J = 32, 16, 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_hist(tpcf, a, b, auto, edges, rank, world):
    na, nb = len(a), len(b)
    _, pairs, cov = tpcf.tpcf_plan_coverage(na, nb, auto, I, JC, J, shard_index=rank, shard_count=world)
    h = np.zeros(len(edges) + 1, dtype=np.uint64)
    for i, j in zip(*np.nonzero(cov)):
        h += oracle.count_cross(a[i:i + 1], b[j:j + 1], edges)
    assert int(h.sum()) == pairs
    return h, cov.astype(np.int64)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1204_6630_gb300 import tpcf
    tpcf.load()
    w = synth.octant_small(seed=4, n=N)
    r = w.rand[:NR]
    res = {}
    for name, a, b, auto in (("dd", w.data, w.data, True), ("dr", w.data, r, False), ("rr", r, r, True)):
        h, cov = _shard_hist(tpcf, a, b, auto, w.edges, rank, world)
        th = torch.from_numpy(h.view(np.int64).copy())
        tc = torch.from_numpy(cov.copy())
        dist.all_reduce(th)
        dist.all_reduce(tc)
        res[name] = (th.numpy().view(np.uint64).copy(), tc.numpy().copy())
    if rank == 0:
        np.save(out, np.array([res], dtype=object), allow_pickle=True)
    dist.destroy_process_group()


def test_two_shards_sum_to_the_unsplit_histograms(tmp_path):
    build.build()
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    res = np.load(out, allow_pickle=True)[0]
    w = synth.octant_small(seed=4, n=N)
    r = w.rand[:NR]
    want = {"dd": oracle.count_auto(w.data, w.edges), "dr": oracle.count_cross(w.data, r, w.edges),
            "rr": oracle.count_auto(r, w.edges)}
    for name in ("dd", "dr", "rr"):
        h, cov = res[name]
        np.testing.assert_array_equal(h, want[name])
        n_a = N if name != "rr" else NR
        n_b = NR if name != "dd" else N
        full = np.triu(np.ones((n_a, n_b), np.int64), 1) if name != "dr" else np.ones((n_a, n_b), np.int64)
        np.testing.assert_array_equal(cov, full)


@pytest.mark.parametrize("world", [2, 3, 7])
def test_shard_item_ranges_partition_every_pair(world):
    build.build()
    from paper_1204_6630_gb300 import tpcf
    for auto, na, nb in ((True, 257, 257), (False, 100, 131)):
        total = np.zeros((na, nb), np.int64)
        items = 0
        for s in range(world):
            it, _, cov = tpcf.tpcf_plan_coverage(na, nb, auto, 64, 32, 16, shard_index=s, shard_count=world)
            total += cov
            items += it
        full = np.triu(np.ones((na, nb), np.int64), 1) if auto else np.ones((na, nb), np.int64)
        np.testing.assert_array_equal(total, full)
        assert items == tpcf.tpcf_plan_coverage(na, nb, auto, 64, 32, 16, with_counts=False)[0]
