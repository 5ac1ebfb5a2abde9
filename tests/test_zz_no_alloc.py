"""The no-allocation auto-count entry point against the regular one, the
oracle and a closed form.

tpcf_count_auto_noalloc serves callers that cannot allocate device memory
(a process whose device memory belongs to another allocator, or a loop that
cannot afford cudaMalloc/cudaFree synchronizing the device).  Its scratch is
a fixed array inside the library shared by every call, so two calls in a row
must each give the same histogram as tpcf_count_auto and as the oracle
(integers, compared exactly as in every other parity test).  All calls run
on one stream.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1204_6630_gb300 import build, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_count_auto_twice_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1204_6630_gb300 import tpcf
    tpcf.load()
    cases = [(synth.octant_small(seed=5, n=3000).data, synth.log_edges(0.01, 10.0, 64)),
             (synth.randoms(2049, synth.Footprint("sphere"), seed=6), np.linspace(0.0, np.pi, 13))]
    with tpcf.Context() as ctx:
        for x, edges in cases:
            want = ctx.count_auto(ctx.catalog(x), ctx.bins(edges))
            dev = torch.from_numpy(x).cuda()
            stream = torch.cuda.current_stream()
            for _ in range(2):
                out = torch.full((len(edges) + 1,), -1, dtype=torch.int64, device="cuda")
                tpcf.tpcf_count_auto_noalloc(dev, edges, out, stream)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64), want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1204_6630_gb300 import tpcf
    edges = np.linspace(0.0, 1.0, tpcf.TPCF_MAX_EDGES + 1)
    dev = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(len(edges) + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.tpcf_count_auto_noalloc(dev, edges, out)
    assert ei.value.status == tpcf.TPCF_EOVERFLOW


def test_noalloc_small_case_equals_the_oracle_twice_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    build.build()
    from paper_1204_6630_gb300 import tpcf
    x = synth.octant_small(seed=11, n=1500).data
    edges = synth.log_edges(0.05, 20.0, 17)
    want = oracle.count_auto(x, edges, threads=4)
    dev = torch.from_numpy(x).cuda()
    for _ in range(2):
        out = torch.full((len(edges) + 1,), -1, dtype=torch.int64, device="cuda")
        tpcf.tpcf_count_auto_noalloc(dev, edges, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64), want)


@pytest.mark.slow
def test_noalloc_one_block_counts_more_than_2_32_pairs_in_one_bin():
    """Edges [0, pi]: every pair is in bin 0 except exact antipodes (theta = pi,
    overflow).  93,200 points give 4.34e9 > 2^32 pairs; with the launch capped at
    one block, that block's shared counter of bin 0 takes all of them, so a
    counter that is never merged before the end of the launch would wrap."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1204_6630_gb300 import tpcf
    rng = np.random.default_rng(3)
    n_rand, k = 93_000, 100
    # random points with z >= 0.01 (no two of them, and none of them with the
    # axis points, are antipodal) plus k copies of (1,0,0) and of (-1,0,0)
    z = rng.uniform(0.01, 1.0, n_rand)
    phi = rng.uniform(0.0, 2 * np.pi, n_rand)
    s_ = np.sqrt(1.0 - z * z)
    pts = np.concatenate([np.stack([s_ * np.cos(phi), s_ * np.sin(phi), z], axis=1),
                          np.tile([[1.0, 0.0, 0.0]], (k, 1)), np.tile([[-1.0, 0.0, 0.0]], (k, 1))])
    n = len(pts)
    total = n * (n - 1) // 2
    assert total > 2 ** 32
    edges = np.array([0.0, np.pi])
    dev = torch.from_numpy(pts).cuda()
    out = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    tpcf.tpcf_debug_noalloc_grid(1)
    try:
        tpcf.tpcf_count_auto_noalloc(dev, edges, out)
        torch.cuda.synchronize()
    finally:
        tpcf.tpcf_debug_noalloc_grid(0)
    h = out.cpu().numpy().view(np.uint64)
    assert int(h[0]) == 0                     # underflow: theta < 0 never
    assert int(h[2]) == k * k                 # overflow: the exact antipodes
    assert int(h[1]) == total - k * k         # everything else, far beyond 2^32
