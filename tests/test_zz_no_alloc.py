"""The no-allocation auto-count entry point against the regular one.

tpcf_count_auto_noalloc serves callers that cannot allocate device memory
(a process whose device memory belongs to another allocator, or a loop that
cannot afford cudaMalloc/cudaFree synchronizing the device).  Its scratch is
a fixed array inside the library shared by every call, so two calls in a row
must each give the same histogram as tpcf_count_auto (integers, compared
exactly as in every other parity test).  This file is collected last.
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
