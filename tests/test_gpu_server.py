"""Job server (tpcf_submit / tpcf_poll / tpcf_cancel).

Every job's histograms must equal the oracle's (small jobs) or a lone
tpcf_correlate call (larger jobs), whatever else runs beside it; the
device-memory budget must serialize jobs that do not fit together and refuse
a job that alone exceeds it; cancel and poll follow their documented states; a
step whose bounded waits expire fails its jobs with TPCF_ETIMEOUT and leaves the
device usable; a job whose bins do not fit the multi-job kernel runs alone.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import build, synth

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
MB = 1 << 20


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1204_6630_gb300 import tpcf
    tpcf.load()
    return tpcf


def job_bytes(nd, nr):
    """The server's admission estimate of one job (kept in step with the library)."""
    def cat(n):
        return ((n + 4095) // 4096 + 1) * 4096 * 60
    n = max(nd, nr)
    p2 = 2048
    while p2 < n:
        p2 *= 2
    return cat(nd) + cat(nr) + n * 24 + p2 * 12 + MB


def octant_job(nd, nr, seed):
    fp = synth.Footprint("octant")
    return synth.clustered(nd, 8, 0.5, fp, seed), synth.randoms(nr, fp, seed + 1000)


def test_jobs_equal_oracle(T):
    edges = synth.linear_edges(0.0, 8.0, 24)
    sizes = [(0, 10), (1, 1), (2, 3), (500, 700), (3000, 1500), (2048, 4097)]
    with T.Context(server_workers=3) as ctx:
        jobs = []
        for k, (nd, nr) in enumerate(sizes):
            d, r = octant_job(nd, nr, seed=10 + k)
            est = k % 2
            jobs.append((ctx.submit(d, r, edges, est), d, r, est))
        for jid, d, r, est in jobs:
            res = ctx.poll(jid, len(edges))
            dd = oracle.count_auto(d, edges, THREADS)
            dr = oracle.count_cross(d, r, edges, THREADS)
            rr = oracle.count_auto(r, edges, THREADS)
            np.testing.assert_array_equal(res["dd"], dd)
            np.testing.assert_array_equal(res["dr"], dr)
            np.testing.assert_array_equal(res["rr"], rr)
            if len(d) >= 2 and len(r) >= 2:
                want = oracle.estimate(dd[1:-1], dr[1:-1], rr[1:-1], len(d), len(r), est)
                np.testing.assert_array_equal(res["w"], want)
            else:
                assert np.all(np.isnan(res["w"]))
            n_d, n_r = len(d), len(r)
            assert res["pairs"] == n_d * (n_d - 1) // 2 + n_d * n_r + n_r * (n_r - 1) // 2
            assert res["latency_ms"] >= res["run_ms"] >= 0 and res["queued_ms"] >= 0


def test_concurrent_jobs_equal_lone_calls(T):
    edges = synth.log_edges(0.01, 10.0, 64)
    specs = [(60000, 120000), (20000, 20000), (90000, 45000), (5000, 200000), (150000, 150000)]
    cats = [octant_job(nd, nr, seed=40 + k) for k, (nd, nr) in enumerate(specs)]
    with T.Context() as ctx:
        alone = [ctx.correlate(d, r, edges) for d, r in cats]
    with T.Context(server_workers=4) as ctx:
        ids = [ctx.submit(d, r, edges) for d, r in cats]
        ids += [ctx.submit(d, r, edges) for d, r in cats]  # the same jobs again, overlapping the first set
        for k, jid in enumerate(ids):
            res = ctx.poll(jid, len(edges))
            want = alone[k % len(cats)]
            for name, w in zip(("dd", "dr", "rr", "w"), want):
                np.testing.assert_array_equal(res[name], w, err_msg=f"job {k} {name}")


def test_budget_serializes_jobs(T):
    edges = synth.linear_edges(0.0, 5.0, 16)
    nd = nr = 100000
    d, r = octant_job(nd, nr, seed=7)
    budget = int(job_bytes(nd, nr) * 1.5)
    with T.Context(server_workers=4, hbm_budget_bytes=budget) as ctx:
        want = ctx.correlate(d, r, edges)
        ids = [ctx.submit(d, r, edges) for _ in range(4)]
        res = [ctx.poll(j, len(edges)) for j in ids]
    spans = sorted((x["submit_ms"] + x["queued_ms"], x["submit_ms"] + x["latency_ms"]) for x in res)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-6, spans  # only one job fits the budget at a time
    for x in res:
        for name, w in zip(("dd", "dr", "rr", "w"), want):
            np.testing.assert_array_equal(x[name], w)


def test_job_over_budget_is_refused(T):
    edges = synth.linear_edges(0.0, 5.0, 16)
    small_d, small_r = octant_job(1000, 1000, seed=8)
    big_d, big_r = octant_job(200000, 200000, seed=9)
    budget = job_bytes(1000, 1000) + 4 * MB
    assert job_bytes(200000, 200000) > budget
    with T.Context(hbm_budget_bytes=budget) as ctx:
        with pytest.raises(T.TpcfError) as e:
            ctx.submit(big_d, big_r, edges)
        assert e.value.status == T.TPCF_EBUDGET
        res = ctx.poll(ctx.submit(small_d, small_r, edges), len(edges))
        np.testing.assert_array_equal(res["dd"], oracle.count_auto(small_d, edges, THREADS))


def test_cancel_and_poll_states(T):
    edges = synth.linear_edges(0.0, 5.0, 16)
    big = octant_job(400000, 400000, seed=11)
    small = octant_job(2000, 2000, seed=12)
    with T.Context(server_workers=1) as ctx:
        first = ctx.submit(*big, edges)
        queued = [ctx.submit(*small, edges) for _ in range(3)]
        ctx.cancel(queued[1])  # still queued behind the big job on the one worker
        res = ctx.poll(queued[1], len(edges), raise_on_error=False)
        assert res["status"] == T.TPCF_ECANCELED and "dd" not in res
        with pytest.raises(T.TpcfError) as e:
            ctx.poll(queued[1], len(edges))
        assert e.value.status == T.TPCF_ENOTFOUND
        with pytest.raises(T.TpcfError) as e:
            ctx.cancel(987654321)
        assert e.value.status == T.TPCF_ENOTFOUND
        want_small = oracle.count_auto(small[0], edges, THREADS)
        for jid in (queued[0], queued[2]):
            np.testing.assert_array_equal(ctx.poll(jid, len(edges))["dd"], want_small)
        assert ctx.poll(first, len(edges))["pairs"] > 0
        # a finished job is not affected by cancel until it is polled
        done = ctx.submit(*small, edges)
        r0 = ctx.poll(done, len(edges), timeout_ms=-1)
        np.testing.assert_array_equal(r0["dd"], want_small)


def test_poll_without_waiting(T):
    edges = synth.linear_edges(0.0, 5.0, 16)
    d, r = octant_job(300000, 300000, seed=13)
    with T.Context(server_workers=1) as ctx:
        jid = ctx.submit(d, r, edges)
        first = ctx.poll(jid, len(edges), timeout_ms=0)
        res = first or ctx.poll(jid, len(edges), timeout_ms=-1)
        assert res["status"] == T.TPCF_OK and res["pairs"] > 0


def test_invalid_jobs(T):
    edges = synth.linear_edges(0.0, 5.0, 16)
    d, r = octant_job(1000, 1000, seed=14)
    with T.Context() as ctx:
        for bad_edges in (edges[::-1], np.array([0.1]), np.array([0.0, 4.0])):
            with pytest.raises(T.TpcfError) as e:
                ctx.submit(d, r, bad_edges)
            assert e.value.status == T.TPCF_EINVAL
        with pytest.raises(T.TpcfError):
            ctx.submit(d, r, edges, estimator=7)
        bad = d.copy()
        bad[17] *= 1.01  # not a unit vector: found when the job runs
        jid = ctx.submit(bad, r, edges)
        res = ctx.poll(jid, len(edges), raise_on_error=False)
        assert res["status"] == T.TPCF_EINVAL
        # the server keeps serving
        ok = ctx.poll(ctx.submit(d, r, edges), len(edges))
        np.testing.assert_array_equal(ok["dr"], oracle.count_cross(d, r, edges, THREADS))


def test_destroy_with_queued_jobs(T):
    edges = synth.linear_edges(0.0, 5.0, 16)
    d, r = octant_job(200000, 200000, seed=15)
    ctx = T.Context(server_workers=1)
    for _ in range(4):
        ctx.submit(d, r, edges)
    ctx.close()  # waits for the running job, drops the queued ones


def test_mixed_sizes_and_bin_sets(T):
    """Serving-style jobs (cap footprints, 20-80 bins, sizes over two decades) in
    flight together use different kernel shapes and shared-memory sizes; each
    result must still equal its lone call."""
    specs = synth.serving_jobs(24, seed=3, nd_min=1e3, nd_max=1.5e5)
    jobs = [synth.materialise_job(s) for s in specs]
    with T.Context() as ctx:
        alone = [ctx.correlate(w.data, w.rand, w.edges) for w in jobs]
    with T.Context(server_workers=6) as ctx:
        ids = [ctx.submit(w.data, w.rand, w.edges) for w in jobs]
        for k, (jid, w) in enumerate(zip(ids, jobs)):
            res = ctx.poll(jid, len(w.edges))
            for name, want in zip(("dd", "dr", "rr", "w"), alone[k]):
                np.testing.assert_array_equal(res[name], want, err_msg=f"job {k} {name}")


def test_a_step_that_times_out_fails_its_jobs_and_the_device_stays_usable(T):
    """With the test hook that leaves each warp's first tile copy unissued, every
    step's bounded waits expire: its jobs finish with TPCF_ETIMEOUT (multi-job
    steps and one-job slices alike), and a fresh server then counts correctly."""
    fp = synth.Footprint("octant")
    small = [octant_job(300 + 50 * k, 600 + 70 * k, 40 + k) for k in range(3)]
    edges = synth.linear_edges(0.0, 10.0, 20)
    with T.Context(flags=T.TPCF_F_TEST_WAIT_TIMEOUT, wait_timeout_us=200_000) as ctx:
        ids = [ctx.submit(d, r, edges) for d, r in small]
        for jid in ids:
            res = ctx.poll(jid, len(edges), raise_on_error=False)
            assert res["status"] == T.TPCF_ETIMEOUT
    d, r = synth.clustered(2000, 8, 0.5, fp, 7), synth.randoms(3000, fp, 8)
    with T.Context() as ctx:
        res = ctx.poll(ctx.submit(d, r, edges), len(edges))
    np.testing.assert_array_equal(res["dd"], oracle.count_auto(d, edges, THREADS))
    np.testing.assert_array_equal(res["dr"], oracle.count_cross(d, r, edges, THREADS))
    np.testing.assert_array_equal(res["rr"], oracle.count_auto(r, edges, THREADS))


def test_a_job_with_too_many_edges_for_the_step_kernel_runs_alone(T):
    """300 bins do not fit the multi-job kernel's shared-memory histograms: that
    job is counted alone by its preparation worker while the others share steps;
    all equal their lone calls."""
    edges_wide = synth.linear_edges(0.0, 3.0, 300)
    edges = synth.linear_edges(0.0, 3.0, 40)
    jobs = [octant_job(4000 + 500 * k, 6000 + 300 * k, 60 + k) for k in range(4)]
    sets = [edges_wide if k == 1 else edges for k in range(len(jobs))]
    with T.Context() as lone:
        want = [lone.correlate(d, r, e) for (d, r), e in zip(jobs, sets)]
    with T.Context() as ctx:
        ids = [ctx.submit(d, r, e) for (d, r), e in zip(jobs, sets)]
        got = [ctx.poll(i, len(e)) for i, e in zip(ids, sets)]
    for k, (g, w_) in enumerate(zip(got, want)):
        for name, a in zip(("dd", "dr", "rr", "w"), w_):
            np.testing.assert_array_equal(g[name], a, err_msg=f"job {k} {name}")


def test_a_small_job_preempts_a_running_large_job(T):
    """A large job's step stops drawing when a small job is ready: the small job,
    submitted while the large one counts, finishes first; both equal lone calls."""
    import time
    edges = synth.linear_edges(0.0, 2.0, 30)
    big = octant_job(700_000, 1_400_000, seed=70)
    small = octant_job(2000, 4000, seed=71)
    with T.Context() as lone:
        want_big = lone.correlate(*big, edges)
        want_small = lone.correlate(*small, edges)
    with T.Context() as ctx:
        jb = ctx.submit(*big, edges)
        time.sleep(0.15)  # the large job is prepared and counting
        js = ctx.submit(*small, edges)
        rs = ctx.poll(js, len(edges))
        rb = ctx.poll(jb, len(edges))
    assert rs["submit_ms"] + rs["latency_ms"] < rb["submit_ms"] + rb["latency_ms"]
    for res, want in ((rb, want_big), (rs, want_small)):
        for name, a in zip(("dd", "dr", "rr", "w"), want):
            np.testing.assert_array_equal(res[name], a)
