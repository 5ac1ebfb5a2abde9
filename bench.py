"""Benchmark: brute-force angular pair counting (DD + DR + RR) on GB300.

Workload (default): the precision-at-scale octant configuration, N_D = N_R =
1,000,000 (data: 70% in 1024 Gaussian clusters of sigma 0.2 deg, 30% uniform;
randoms uniform on the octant), 64 log-spaced bins over 0.01-10 deg, seed 0.
Synthetic stand-in for the paper's MICE catalogs.

One step = the whole hot path on device-resident binary64 coordinates:
catalog preparation of D and R (validation, spatial sort, FP32/binary64
copies), bin thresholds, one fused DD/DR/RR counting launch, the finalize
kernels, and the Landy-Szalay estimate.  `value` is pairs/s over the K timed
steps (CUDA events, max over ranks).  `e2e` repeats the step through the
host-array call tpcf_correlate with the catalogs in pinned host memory (copies
included).  The roofline is that of the counting kernel: 3 FP32 pipe lane
operations per pair (3 FFMA, the range offset folded into the first), counted
as 6 flops, against the FP32 peak derived from the device's SM count x 128
lanes x 2 flops x the maximum SM clock (nvidia-smi), with the fraction at the
clock sampled under load and against the measured FMA-chain throughput
(tpcf_fp32_peak) beside it.  The line also carries the all-binary64 kernel on
the same catalogs (`fp64_plain`) and one launch with spatial pruning
(`pruning`, the opt-in TPCF_F_PRUNE flag: same histograms, pairs covered per
second); neither is the brute-force headline.  After the timed region, compact
records of the other workloads (skipped with --no-extras): `large` (one fused
launch of the 4M + 8M full-sphere problem with its roofline fraction, a
40,000-point oracle check and near-edge pairs), `jackknife` (the 512-patch
graph against separate calls) and `serving` (a 100-job stream against
one-at-a-time calls: throughput and p50/p99 latency).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Other workloads (one JSON line each, not the headline line):
  --workload jackknife  2,000,000 data + 4,000,000 random octant points in 512
                        patches of lognormal size (1k-200k), 40 linear bins
                        0-5 deg: per-patch DD/DR/RR as one captured graph
                        (autotuned shape) against 1,536 separate launches,
                        and the leave-one-out jackknife of the full catalogs
                        (brute force and pruned);
  --workload serving    a Poisson stream of --jobs jobs (N_D log-uniform in
                        [1e3, 1e6], N_R = 2 N_D, caps of 5-30 deg, 20-80
                        linear bins over 0-2 deg) through the job server
                        under a 120 GB budget, against one-at-a-time calls:
                        p50/p99 latency and throughput (also with pruning);
  --workload box3d      the 3-D variant: 1,000,000 clustered + 1,000,000 uniform
                        points in a box of side 1000, 30 log distance bins
                        0.5-50 (subsample checked against the oracle);
  --workload large      4,000,000 clustered data + 8,000,000 random points on
                        the full sphere, 80 log bins 0.005-2 deg, with exact
                        counts checked against the oracle on a 100,000-point
                        random subsample of each catalog.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s (DD+DR+RR)"
UNIT = "pairs/s"
FLOPS_PER_PAIR = 6            # 3 FP32 pipe lane-ops (3 FFMA), FMA convention
L2_FLUSH_BYTES = 256 << 20


def workload_config(n: int, bins: int) -> dict:
    return {"workload": f"octant_precision: N_D=N_R={n:,} (data 70% in 1024 clusters sigma 0.2 deg, "
                        f"randoms uniform), {bins} log bins 0.01-10 deg, seed 0",
            "nd": n, "nr": n, "nbins": bins,
            "pairs_per_step": None,
            "l2": "256 MB buffer rewritten between timed steps",
            "step": "catalog prep (D, R) + thresholds + fused DD/DR/RR launch + finalize + estimate"}


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(w, n_sample: int, threads: int, hists: bool = False):
    """Time the oracle on the first n_sample points of D and R (DD + DR + RR);
    with ``hists`` also return its (DD, DR, RR) histograms."""
    import oracle
    d, r = w.data[:n_sample], w.rand[:n_sample]
    t0 = time.perf_counter()
    dd, dr, rr, _ = oracle.correlation(d, r, w.edges, threads=threads)
    dt = time.perf_counter() - t0
    pairs = n_sample * (n_sample - 1) + n_sample * n_sample
    if hists:
        return pairs / dt, dt, pairs, (dd, dr, rr)
    return pairs / dt, dt, pairs


def near_edge_count(d, r, edges, threads: int, tol: float = 1e-12) -> int:
    """Oracle pairs (DD, RR, DR of the sample) whose angle is within tol of an edge:
    the only pairs whose bin may depend on the arc-cosine that decides it."""
    import oracle
    return sum(oracle.near_edge_pairs(a, b, edges, auto, tol=tol, threads=threads)[0]
               for auto, a, b in ((True, d, None), (True, r, None), (False, d, r)))


def roofline_peaks(local: int, clocks: dict):
    """Derived FP32 peak (device SM count x 128 lanes x 2 flops x the maximum SM
    clock nvidia-smi reports), the same at the median clock sampled under load,
    and the measured FMA-chain throughput (scalar and packed)."""
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    med_mhz = clocks.get("sm_mhz") or max_mhz
    derived = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    at_clock = sms * 128 * 2 * med_mhz * 1e6 / 1e12
    return sms, max_mhz, med_mhz, derived, at_clock


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_1204_6630_gb300 import synth
    w = synth.octant_precision(seed=0, n=args.n)
    cores = os.cpu_count() or 1
    n_s = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample(w, min(n_s, 2000), cores)
    vals, times, pairs = [], [], 0
    for _ in range(args.steps):
        v, dt, pairs = oracle_sample(w, n_s, cores)
        vals.append(v)
        times.append(dt)
    value = sum(pairs for _ in vals) / sum(times)
    sample = (f"first {n_s:,} points of D and of R of the {args.n:,}-point workload, all 64 bins; "
              f"DD+DR+RR = {pairs:,} pairs per step")
    cfg = workload_config(args.n, len(w.edges) - 1)
    cfg["pairs_per_step"] = pairs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1204_6630_gb300 import synth, tpcf

    w = synth.octant_precision(seed=0, n=args.n)
    nd, nr, nbins = len(w.data), len(w.rand), len(w.edges) - 1
    pairs = nd * (nd - 1) // 2 + nr * (nr - 1) // 2 + nd * nr
    dev_d = torch.from_numpy(w.data).cuda()
    dev_r = torch.from_numpy(w.rand).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = tpcf.Context(device=local, shard_index=rank if world > 1 else 0,
                       shard_count=world if world > 1 else 0)

    def step():
        cd = ctx.catalog(dev_d, stream)
        cr = ctx.catalog(dev_r, stream)
        b = ctx.bins(w.edges)
        (dd, dr, rr), st = ctx.count_all(cd, cr, b, stream, stats=True)
        if world > 1:
            import torch.distributed as dist
            t = torch.from_numpy(np.stack([dd, dr, rr]).view(np.int64)).cuda()
            dist.all_reduce(t)
            dd, dr, rr = t.cpu().numpy().view(np.uint64)
        wt = tpcf.tpcf_estimate(dd[1:-1], dr[1:-1], rr[1:-1], nd, nr)
        ctx.free(cd)
        ctx.free(cr)
        ctx.free(b)
        return st, (dd, dr, rr, wt)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
        flush.zero_()
    barrier()
    launches0 = tpcf.tpcf_kernel_launches(ctx.handle)
    kernel_ms = []
    with ClockSampler(local) as clocks:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for k in range(args.steps):
            st, out = step()
            kernel_ms.append(st["kernel_ms"])
            if k + 1 < args.steps:
                flush.zero_()
        ev1.record(stream)
        barrier()
        elapsed_ms = ev0.elapsed_time(ev1)
    launches = tpcf.tpcf_kernel_launches(ctx.handle) - launches0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    dd, dr, rr, wt = out
    assert int(dd.sum()) == nd * (nd - 1) // 2 and int(dr.sum()) == nd * nr and int(rr.sum()) == nr * (nr - 1) // 2

    # ---- end to end through the host-array C call (pinned inputs, copies inside)
    pin_d = torch.from_numpy(w.data).pin_memory()
    pin_r = torch.from_numpy(w.rand).pin_memory()
    e2e = None
    if world == 1:
        for _ in range(max(1, args.warmup // 2)):
            ctx.correlate(pin_d.numpy(), pin_r.numpy(), w.edges)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.correlate(pin_d.numpy(), pin_r.numpy(), w.edges)
            flush.zero_()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": pairs * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(w.data.nbytes + w.rand.nbytes + w.edges.nbytes),
               "d2h_bytes_per_step": int(3 * (nbins + 2) * 8 + 8 * 8)}
    else:
        # every rank counts its shard through the host-array call (the whole
        # catalogs go up on each rank), the shards' histograms are summed; the
        # slowest rank's time counts (a failure here leaves e2e empty, never the line)
        import torch.distributed as dist
        try:
            ctx.correlate(pin_d.numpy(), pin_r.numpy(), w.edges)
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                edd, edr, err_, _ = ctx.correlate(pin_d.numpy(), pin_r.numpy(), w.edges)
                th = torch.from_numpy(np.stack([edd, edr, err_]).view(np.int64)).cuda()
                dist.all_reduce(th)
            barrier()
            t = torch.tensor([time.perf_counter() - t0], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
            same = all(np.array_equal(x, y) for x, y in zip(th.cpu().numpy().view(np.uint64), (dd, dr, rr)))
            e2e = {"value": pairs * args.steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": int(world * (w.data.nbytes + w.rand.nbytes + w.edges.nbytes)),
                   "d2h_bytes_per_step": int(world * (3 * (nbins + 2) * 8 + 8 * 8)),
                   "histograms_identical": same}
        except Exception as exc:  # reported, not fatal
            e2e = {"value": None, "unit": UNIT, "error": f"{type(exc).__name__}: {exc}"}

    # ---- the all-binary64 kernel on the same resident catalogs: one launch
    fp64 = None
    if world == 1 and not args.no_fp64:
        with tpcf.Context(device=local, precision=tpcf.TPCF_PLAIN_FP64) as c64:
            cd, cr, b = c64.catalog(dev_d, stream), c64.catalog(dev_r, stream), c64.bins(w.edges)
            (pdd, pdr, prr), st64 = c64.count_all(cd, cr, b, stream, stats=True)
        same = all(np.array_equal(a, c) for a, c in zip((pdd, pdr, prr), (dd, dr, rr)))
        fp64 = {"kernel": "count_kernel, all-binary64 mode (fused DD/DR/RR)",
                "kernel_ms": st64["kernel_ms"], "pairs_per_s": st64["pairs"] / st64["kernel_ms"] * 1e3,
                "screen_speedup": st64["kernel_ms"] / statistics.mean(kernel_ms),
                "histograms_identical": same}
        assert same, "FP32 screen + recheck and all-binary64 kernels disagree"

    # ---- spatial pruning (opt-in flag, not the brute-force headline): one launch
    # on the same resident catalogs, histograms compared with the brute force;
    # skipped slots include padding and masked (diagonal) slots, so their ratio to
    # the covered pairs can exceed the fraction of pairs skipped (or even 1)
    prune = None
    if world == 1 and not args.no_prune:
        with tpcf.Context(device=local, flags=tpcf.TPCF_F_PRUNE) as cp:
            cd, cr, b = cp.catalog(dev_d, stream), cp.catalog(dev_r, stream), cp.bins(w.edges)
            cp.count_all(cd, cr, b, stream)  # warm-up
            (qdd, qdr, qrr), stp = cp.count_all(cd, cr, b, stream, stats=True)
        prune = {"flag": "TPCF_F_PRUNE", "kernel_ms": stp["kernel_ms"],
                 "pairs_covered_per_s": stp["pairs"] / stp["kernel_ms"] * 1e3,
                 "pair_slots_skipped": stp["pruned_pairs"],
                 "skipped_slots_per_pair": stp["pruned_pairs"] / stp["pairs"],
                 "histograms_identical": all(np.array_equal(a, c) for a, c in zip((qdd, qdr, qrr), (dd, dr, rr)))}
        assert prune["histograms_identical"], "pruned and brute-force histograms disagree"

    # measured FP32 FMA throughput (the roofline's measured denominator), GPU otherwise idle
    peak_meas = None
    if rank == 0:
        pk_s = tpcf.tpcf_fp32_peak(local, packed=False)
        pk_p = tpcf.tpcf_fp32_peak(local, packed=True)
        peak_meas = {"value": max(pk_s, pk_p), "fma_f32": pk_s, "fma_f32x2": pk_p,
                     "source": "tpcf_fp32_peak: 16 independent FMA chains per thread, 4 x 512 threads per SM, "
                               "best of 5 launches (CUDA events)"}

    cpu = None
    sub_parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        # single-threaded oracle (the baseline), then the same oracle on every host core
        v1, dt1, sp1 = oracle_sample(w, args.cpu_sample_1t, 1)
        v, dt, sp, ohist = oracle_sample(w, args.cpu_sample, cores, hists=True)
        cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {args.cpu_sample_1t:,} points of D and of R, DD+DR+RR = {sp1:,} pairs, "
                         f"{dt1:.1f} s on one host thread",
               "multi_thread": {"value": v, "unit": UNIT, "threads": cores,
                                "sample": f"first {args.cpu_sample:,} points of D and of R, DD+DR+RR = "
                                          f"{sp:,} pairs, {dt:.1f} s"}}
        # the GPU path on the same sample, compared with the oracle's histograms
        cs_d, cs_r = ctx.catalog(w.data[:args.cpu_sample]), ctx.catalog(w.rand[:args.cpu_sample])
        gs = ctx.count_all(cs_d, cs_r, ctx.bins(w.edges))
        sub_parity = {"points_per_catalog": args.cpu_sample,
                      "identical_to_oracle": all(np.array_equal(a, b) for a, b in zip(gs, ohist)),
                      "near_edge_pairs": near_edge_count(w.data[:args.cpu_sample], w.rand[:args.cpu_sample],
                                                         w.edges, cores),
                      "near_edge_tol_rad": 1e-12}

    kern_s = statistics.mean(kernel_ms) / 1e3
    achieved = st["pairs"] * FLOPS_PER_PAIR / kern_s / 1e12   # this rank's launch
    traffic = None
    prof = os.path.join(ROOT, "profiles", "count_kernel_traffic.json")
    if os.path.exists(prof):
        # the recorded DRAM bytes count only while the kernel source is the one they were taken from
        try:
            import hashlib
            rec = json.load(open(prof))
            src = os.path.join(ROOT, "paper_1204_6630_gb300", "csrc", "count.cu")
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            if rec.get("kernel_source_sha256_16") == sha and args.n == 1_000_000:
                traffic = rec.get("dram_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    cfg = workload_config(args.n, nbins)
    cfg["pairs_per_step"] = pairs
    cfg["parallelism"] = f"shards{world}" if world > 1 else "single"
    csum = clocks.summary()
    sms, max_mhz, med_mhz, peak_derived, peak_clock = roofline_peaks(local, csum)
    if peak_meas:
        peak_meas["frac"] = achieved / peak_meas["value"]
    line = {
        "metric": METRIC, "value": pairs * args.steps / (elapsed_ms / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32", "precision": "FP32 screen + binary64 guard-band recheck, uint64 counts",
        "data": "synthetic", "config": cfg,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_derived, "unit": "TFLOP/s",
                     "frac": achieved / peak_derived, "traffic": traffic,
                     "kernel": "count_kernel (screen, fused DD/DR/RR)",
                     "kernel_ms": statistics.mean(kernel_ms),
                     "peak_source": f"derived: {sms} SMs (device) x 128 FP32 lanes x 2 flops x {max_mhz:.0f} MHz "
                                    "(maximum SM clock, nvidia-smi); MEASURED_PEAKS.json has no FP32 entry",
                     "peak_at_sampled_clock": {"value": peak_clock, "sm_mhz": med_mhz,
                                               "frac": achieved / peak_clock},
                     "peak_measured": peak_meas},
        "band": {"pairs": st["band_pairs"], "fraction": st["band_pairs"] / max(1, st["pairs"]),
                 "fp32_mismatch": st["band_mismatch"]},
        "fp64_plain": fp64,
        "pruning": prune,
        "subsample_parity": sub_parity,
        "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches,
        "clocks": csum,
    }
    ctx.close()
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(extras(peak_meas["value"] if peak_meas else None))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def extras(peak_meas) -> dict:
    """Compact records of the other workloads, after the timed region of the
    headline: the 4M + 8M full-sphere launch (roofline, 40k-point oracle check,
    near-edge pairs), the 512-patch jackknife graph against separate calls, and a
    100-job serving stream against one-at-a-time calls."""
    lg = large_record(1, 1, 40_000, prune=False, peak_meas=peak_meas)
    jk = jackknife_record(3, 1, loo=False)
    sv = serving_record(100, 0, pruned=False)
    return {
        "large": {"workload": lg["config"]["workload"], "pairs": lg["config"]["pairs_per_step"],
                  "kernel_ms": lg["ms_per_step"], "pairs_per_s": lg["value"],
                  "frac": lg["roofline"]["frac"], "frac_of_measured": lg["roofline"]["frac_of_measured"],
                  "band_pairs": lg["band"]["pairs"],
                  "subsample_points": lg["subsample_parity"]["points_per_catalog"],
                  "subsample_identical_to_oracle": lg["subsample_parity"]["identical_to_oracle"],
                  "near_edge_pairs": lg["subsample_parity"]["near_edge_pairs"],
                  "clocks": lg["clocks"]},
        "jackknife": {"workload": jk["config"]["workload"], "patches": jk["config"]["patches"],
                      "pairs": jk["config"]["pairs_per_step"], "graph_ms": jk["graph"]["ms"],
                      "separate_ms": jk["separate"]["ms"], "speedup_vs_separate": jk["speedup_vs_separate"],
                      "histograms_identical": jk["histograms_identical"]},
        "serving": {"workload": sv["config"]["workload"], "jobs": sv["config"]["jobs"],
                    "throughput_vs_serial": sv["throughput_vs_serial"],
                    "serial_s": sv["serial"]["s"], "served_s": sv["served_burst"]["s"],
                    "latency_s_poisson": {"served": sv["served_poisson"]["latency_s"],
                                          "serial": sv["serial"]["latency_s_at_poisson"]},
                    "arrivals": sv["config"]["arrivals"],
                    "results_identical_to_lone_calls": sv["results_identical_to_lone_calls"]},
    }


def run_count_only(args):
    """One warm-up and one fused DD/DR/RR launch on the octant workload of
    args.count_only points per catalog (the command the profiles use)."""
    from paper_1204_6630_gb300 import synth, tpcf
    w = synth.octant_precision(seed=0, n=args.count_only)
    with tpcf.Context() as ctx:
        d, r, b = ctx.catalog(w.data), ctx.catalog(w.rand), ctx.bins(w.edges)
        for _ in range(2):
            _, st = ctx.count_all(d, r, b, stats=True)
        print(json.dumps({"n": args.count_only, "kernel_ms": st["kernel_ms"],
                          "pairs_per_s": st["pairs"] / st["kernel_ms"] * 1e3, "band_pairs": st["band_pairs"]}))
    return 0


# ----------------------------------------------------------------------------- other workloads
def _quantiles(xs):
    a = np.sort(np.asarray(xs, dtype=np.float64))
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "max": float(a[-1])}


def jackknife_record(steps: int, warmup: int, loo: bool = True) -> dict:
    """Per-patch DD/DR/RR of 512 patches: one captured graph vs separate launches
    (and, with ``loo``, the leave-one-out jackknife, brute force and pruned)."""
    import torch
    from paper_1204_6630_gb300 import synth, tpcf
    d, r, doff, roff = synth.jackknife_patches(seed=0)
    edges = synth.linear_edges(0.0, 5.0, 40)
    nd_p, nr_p = np.diff(doff), np.diff(roff)
    pairs = int(sum(n * (n - 1) // 2 + m * (m - 1) // 2 + n * m for n, m in zip(nd_p, nr_p)))
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    with tpcf.Context(flags=tpcf.TPCF_F_AUTOTUNE) as ctx:
        cd = ctx.catalog(torch.from_numpy(d).cuda(), stream, offsets=doff)
        cr = ctx.catalog(torch.from_numpy(r).cuda(), stream, offsets=roff)
        b = ctx.bins(edges)
        t0 = time.perf_counter()
        g = ctx.graph(tpcf.TPCF_GRAPH_PATCHES, cd, cr, b)  # autotunes, then captures
        torch.cuda.synchronize()
        create_s = time.perf_counter() - t0
        for _ in range(warmup):
            g.launch(stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        graph_ms = []
        for _ in range(steps):
            flush.zero_()
            ev[0].record(stream)
            g.launch(stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            graph_ms.append(ev[0].elapsed_time(ev[1]))
        st = g.stats()
        batched = g.out.cpu().numpy().view(np.uint64).copy()

        # separate launches: one catalog pair per patch (prepared beforehand), 3 calls per patch
        sub = []
        for p in range(len(nd_p)):
            sub.append((ctx.catalog(torch.from_numpy(d[doff[p]:doff[p + 1]]).cuda(), stream),
                        ctx.catalog(torch.from_numpy(r[roff[p]:roff[p + 1]]).cuda(), stream)))
        sep_out = torch.empty((len(nd_p), 3, len(edges) + 1), dtype=torch.int64, device="cuda")

        def separate():
            for p, (cdp, crp) in enumerate(sub):
                ctx.count_auto(cdp, b, stream, out=sep_out[p, 0])
                ctx.count_cross(cdp, crp, b, stream, out=sep_out[p, 1])
                ctx.count_auto(crp, b, stream, out=sep_out[p, 2])

        separate()
        sep_ms = []
        for _ in range(max(1, steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            ev[0].record(stream)
            separate()
            ev[1].record(stream)
            torch.cuda.synchronize()
            sep_ms.append(ev[0].elapsed_time(ev[1]))
        same = np.array_equal(sep_out.cpu().numpy().view(np.uint64), batched)
        assert same and st["pairs"] == pairs
        for o in sub:
            ctx.free(o[0])
            ctx.free(o[1])
        if loo:
            # leave-one-out jackknife of the full catalogs over the same patches
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loo_h, w_loo, cov, jst = ctx.jackknife(cd, cr, b, stream, stats=True)
            loo_s = time.perf_counter() - t0
    gm, sm = statistics.median(graph_ms), statistics.median(sep_ms)
    rec = {
        "mode": "jackknife", "metric": METRIC, "value": pairs / gm * 1e3, "unit": UNIT,
        "steps": steps, "warmup": warmup, "ms_per_step": gm, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "octant jackknife: N_D=2,000,000 (1024 clusters sigma 0.2 deg), N_R=4,000,000, "
                               "512 patches lognormal 1k-200k, 40 linear bins 0-5 deg, seed 0",
                   "patches": int(len(nd_p)), "pairs_per_step": pairs,
                   "patch_nd": {"min": int(nd_p.min()), "median": float(np.median(nd_p)), "max": int(nd_p.max())},
                   "l2": "256 MB buffer rewritten before each timed launch"},
        "graph": {"ms": gm, "pairs_per_s": pairs / gm * 1e3, "create_s": create_s,
                  "launches_per_replay": st["launches"], "band_pairs": st["band_pairs"]},
        "separate": {"ms": sm, "pairs_per_s": pairs / sm * 1e3, "calls": 3 * int(len(nd_p)),
                     "launches": 3 * 2 * int(len(nd_p))},
        "speedup_vs_separate": sm / gm, "histograms_identical": same}
    if loo:
        # the same leave-one-out jackknife with spatial pruning (opt-in): most block
        # pairs of the full catalogs are farther apart than the 5 deg range
        with tpcf.Context(flags=tpcf.TPCF_F_PRUNE) as cq:
            qd, qr, qb = cq.catalog(d, offsets=doff), cq.catalog(r, offsets=roff), cq.bins(edges)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            qloo, qw, qcov, qst = cq.jackknife(qd, qr, qb, stream, stats=True)
            qloo_s = time.perf_counter() - t0
        loo_same = (np.array_equal(qloo, loo_h) and np.array_equal(qw, w_loo, equal_nan=True)
                    and np.array_equal(qcov, cov, equal_nan=True))
        assert loo_same, "pruned and brute-force leave-one-out results disagree"
        rec["leave_one_out"] = {"s": loo_s, "kernel_ms": jst["kernel_ms"], "pairs": jst["pairs"],
                                "pairs_per_s": jst["pairs"] / loo_s,
                                "what": "DD/DR/RR of the catalogs without each patch (512 resamplings), w and "
                                        "its covariance: one launch over every pair of the full catalogs"}
        rec["leave_one_out_pruned"] = {"flag": "TPCF_F_PRUNE", "s": qloo_s, "kernel_ms": qst["kernel_ms"],
                                       "pairs_covered_per_s": qst["pairs"] / qloo_s,
                                       "skipped_slots_per_pair": qst["pruned_pairs"] / max(1, qst["pairs"]),
                                       "identical_to_brute_force": loo_same}
    return rec


def run_jackknife(args):
    print(json.dumps(jackknife_record(args.steps, args.warmup)))
    return 0


def serving_record(njobs: int, workers: int, pruned: bool = True) -> dict:
    """Poisson job stream through the job server vs one-at-a-time calls (and, with
    ``pruned``, the same with spatial pruning)."""
    import concurrent.futures as cf
    import torch
    from paper_1204_6630_gb300 import synth, tpcf
    specs = synth.serving_jobs(njobs, seed=0)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        jobs = list(ex.map(synth.materialise_job, specs))
    gen_s = time.perf_counter() - t0
    pairs = [w.pairs for w in jobs]
    total_pairs = sum(pairs)
    budget = 120 << 30

    # serial: one synchronous call per job, in arrival order
    with tpcf.Context() as ctx:
        for w in jobs[:3]:
            ctx.correlate(w.data, w.rand, w.edges)
        torch.cuda.synchronize()
        service = []
        serial_res = []
        t0 = time.perf_counter()
        for w in jobs:
            t1 = time.perf_counter()
            serial_res.append(ctx.correlate(w.data, w.rand, w.edges))
            service.append(time.perf_counter() - t1)
        serial_s = time.perf_counter() - t0
    rate = 0.8 * len(jobs) / serial_s   # Poisson arrival rate: 80% of the serial job rate
    gaps = np.random.default_rng(1).exponential(1.0 / rate, len(jobs))
    arrivals = np.cumsum(gaps) - gaps[0]
    # the serial system under the same arrivals (FIFO, measured service times)
    done, serial_lat = 0.0, []
    for a, sv in zip(arrivals, service):
        done = max(done, a) + sv
        serial_lat.append(done - a)

    def serve(at, flags=0):
        with tpcf.Context(hbm_budget_bytes=budget, server_workers=workers, flags=flags) as ctx:
            ctx.poll(ctx.submit(jobs[0].data, jobs[0].rand, jobs[0].edges), len(jobs[0].edges))
            start = time.perf_counter()
            ids = []
            for k, w in enumerate(jobs):
                wait = start + at[k] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                ids.append((ctx.submit(w.data, w.rand, w.edges), time.perf_counter() - start))
            res = [ctx.poll(j, len(w.edges)) for (j, _), w in zip(ids, jobs)]
            span = max(s + x["latency_ms"] / 1e3 for (_, s), x in zip(ids, res))
        lat = [x["latency_ms"] / 1e3 + (s - at[k]) for k, ((_, s), x) in enumerate(zip(ids, res))]
        return res, span, lat

    burst_res, burst_span, burst_lat = serve(np.zeros(len(jobs)))
    pois_res, pois_span, pois_lat = serve(arrivals)
    same = all(np.array_equal(x[n], y[i]) for x, y in zip(burst_res, serial_res)
               for i, n in enumerate(("dd", "dr", "rr"))) and \
        all(np.array_equal(x[n], y[i]) for x, y in zip(pois_res, serial_res)
            for i, n in enumerate(("dd", "dr", "rr")))
    assert same, "served results differ from lone calls"
    nd = np.array([len(w.data) for w in jobs])
    rec = {
        "mode": "serving", "metric": "jobs/s and pairs/s; p50/p99 job latency", "value": total_pairs / burst_span,
        "unit": UNIT, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serving: {len(jobs)} jobs, N_D log-uniform [1e3, 1e6], N_R = 2 N_D, caps 5-30 deg, "
                               "128 clusters sigma 0.5 deg, 20-80 linear bins 0-2 deg, seed 0",
                   "jobs": len(jobs), "pairs_total": total_pairs, "nd_median": float(np.median(nd)),
                   "hbm_budget_gb": budget / 2**30, "workers": workers, "generation_s": gen_s,
                   "arrival_rate_hz": rate, "arrivals": "Poisson at 0.8 x the serial job rate"},
        "serial": {"s": serial_s, "jobs_per_s": len(jobs) / serial_s, "pairs_per_s": total_pairs / serial_s,
                   "latency_s_at_poisson": _quantiles(serial_lat)},
        "served_burst": {"s": burst_span, "jobs_per_s": len(jobs) / burst_span,
                         "pairs_per_s": total_pairs / burst_span, "latency_s": _quantiles(burst_lat)},
        "served_poisson": {"s": pois_span, "jobs_per_s": len(jobs) / pois_span,
                           "pairs_per_s": total_pairs / pois_span, "latency_s": _quantiles(pois_lat)},
        "throughput_vs_serial": serial_s / burst_span, "results_identical_to_lone_calls": same}
    if pruned:
        # the same stream with spatial pruning (opt-in flag): one-at-a-time and served
        with tpcf.Context(flags=tpcf.TPCF_F_PRUNE) as ctx:
            ctx.correlate(jobs[0].data, jobs[0].rand, jobs[0].edges)
            t0 = time.perf_counter()
            pser_res = [ctx.correlate(w.data, w.rand, w.edges) for w in jobs]
            pserial_s = time.perf_counter() - t0
        pburst_res, pburst_span, pburst_lat = serve(np.zeros(len(jobs)), tpcf.TPCF_F_PRUNE)
        psame = all(np.array_equal(x[n], y[i]) for x, y in zip(pburst_res, serial_res)
                    for i, n in enumerate(("dd", "dr", "rr"))) and \
            all(np.array_equal(x[i], y[i]) for x, y in zip(pser_res, serial_res) for i in range(3))
        assert psame, "pruned results differ from brute-force lone calls"
        rec["pruned"] = {"flag": "TPCF_F_PRUNE",
                         "serial": {"s": pserial_s, "pairs_per_s": total_pairs / pserial_s},
                         "served_burst": {"s": pburst_span, "pairs_per_s": total_pairs / pburst_span,
                                          "latency_s": _quantiles(pburst_lat)},
                         "throughput_vs_pruned_serial": pserial_s / pburst_span,
                         "throughput_vs_brute_force_serial": serial_s / pburst_span,
                         "results_identical_to_brute_force": psame}
    return rec


def run_serving(args):
    print(json.dumps(serving_record(args.jobs, args.workers)))
    return 0


def large_record(steps: int, warmup: int, sub: int, prune: bool = True, peak_meas=None) -> dict:
    """4M + 8M full-sphere points: timed fused launch, oracle check (and near-edge
    pairs) on a random subsample of each catalog; with ``prune`` also one launch
    with spatial pruning.  peak_meas: the measured FP32 peak (TFLOP/s), if taken."""
    import torch
    import oracle
    from paper_1204_6630_gb300 import synth, tpcf
    w = synth.sphere_large(seed=0)
    nd, nr = len(w.data), len(w.rand)
    pairs = w.pairs
    stream = torch.cuda.current_stream()
    with tpcf.Context() as ctx:
        cd = ctx.catalog(torch.from_numpy(w.data).cuda(), stream)
        cr = ctx.catalog(torch.from_numpy(w.rand).cuda(), stream)
        b = ctx.bins(w.edges)
        for _ in range(warmup):
            ctx.count_all(cd, cr, b, stream)
        kms = []
        with ClockSampler(0) as clocks:
            for _ in range(steps):
                (dd, dr, rr), st = ctx.count_all(cd, cr, b, stream, stats=True)
                kms.append(st["kernel_ms"])
        assert int(dd.sum()) == nd * (nd - 1) // 2 and int(dr.sum()) == nd * nr and int(rr.sum()) == nr * (nr - 1) // 2
        # subsample parity
        g = np.random.default_rng(7)
        ds = w.data[np.sort(g.choice(nd, sub, replace=False))]
        rs = w.rand[np.sort(g.choice(nr, sub, replace=False))]
        sdd, sdr, srr = ctx.count_all(ctx.catalog(ds), ctx.catalog(rs), b)
        ctx.free(cd)
        ctx.free(cr)
    pr = None
    if prune:
        # the same counts with spatial pruning (opt-in; not the brute-force headline)
        with tpcf.Context(flags=tpcf.TPCF_F_PRUNE) as cq:
            qd = cq.catalog(torch.from_numpy(w.data).cuda(), stream)
            qr = cq.catalog(torch.from_numpy(w.rand).cuda(), stream)
            qb = cq.bins(w.edges)
            cq.count_all(qd, qr, qb, stream)
            (qdd, qdr, qrr), qst = cq.count_all(qd, qr, qb, stream, stats=True)
        pr = {"flag": "TPCF_F_PRUNE", "kernel_ms": qst["kernel_ms"],
              "pairs_covered_per_s": qst["pairs"] / qst["kernel_ms"] * 1e3,
              "skipped_slots_per_pair": qst["pruned_pairs"] / qst["pairs"],
              "histograms_identical": all(np.array_equal(x, y) for x, y in zip((qdd, qdr, qrr), (dd, dr, rr)))}
        assert pr["histograms_identical"], "pruned and brute-force histograms disagree"
    t0 = time.perf_counter()
    cores = os.cpu_count() or 1
    odd = oracle.count_auto(ds, w.edges, cores)
    odr = oracle.count_cross(ds, rs, w.edges, cores)
    orr = oracle.count_auto(rs, w.edges, cores)
    oracle_s = time.perf_counter() - t0
    same = np.array_equal(odd, sdd) and np.array_equal(odr, sdr) and np.array_equal(orr, srr)
    assert same, "subsample histograms differ from the oracle"
    km = statistics.mean(kms)
    ach = pairs * FLOPS_PER_PAIR / (km / 1e3) / 1e12
    csum = clocks.summary()
    sms, max_mhz, _, peak_derived, _ = roofline_peaks(0, csum)
    rec = {
        "mode": "large", "metric": METRIC, "value": pairs / km * 1e3, "unit": UNIT, "steps": steps,
        "warmup": warmup, "ms_per_step": km, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sphere_large: N_D=4,000,000 (4096 clusters sigma 0.1 deg), N_R=8,000,000 uniform, "
                               "full sphere, 80 log bins 0.005-2 deg, seed 0", "pairs_per_step": pairs,
                   "timed": "fused DD/DR/RR counting launch + finalize on resident catalogs (CUDA events)"},
        "roofline": {"bound": "alu", "achieved": ach, "peak": peak_derived, "unit": "TFLOP/s",
                     "frac": ach / peak_derived,
                     "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flops x {max_mhz:.0f} MHz",
                     "peak_measured": peak_meas,
                     "frac_of_measured": ach / peak_meas if peak_meas else None},
        "band": {"pairs": st["band_pairs"], "fraction": st["band_pairs"] / pairs,
                 "fp32_mismatch": st["band_mismatch"]},
        "subsample_parity": {"points_per_catalog": sub, "identical_to_oracle": same,
                             "oracle_s": oracle_s, "oracle_threads": cores,
                             "near_edge_pairs": near_edge_count(ds, rs, w.edges, cores),
                             "near_edge_tol_rad": 1e-12},
        "clocks": csum}
    if pr:
        rec["pruning"] = pr
    return rec


def run_large(args):
    print(json.dumps(large_record(args.steps, args.warmup, args.sub)))
    return 0


def run_box3d(args):
    """3-D variant: 1M clustered + 1M uniform points in a box of side 1000, 30 log
    distance bins 0.5-50; fused DD/DR/RR launch on resident catalogs."""
    import torch
    import oracle
    from paper_1204_6630_gb300 import synth, tpcf
    w = synth.box_precision(seed=0, n=args.n)
    nd, nr = len(w.data), len(w.rand)
    pairs = w.pairs
    stream = torch.cuda.current_stream()
    with tpcf.Context() as ctx:
        cd = ctx.catalog3d(torch.from_numpy(w.data).cuda(), stream)
        cr = ctx.catalog3d(torch.from_numpy(w.rand).cuda(), stream)
        b = ctx.bins3d(w.edges)
        for _ in range(args.warmup):
            ctx.count_all(cd, cr, b, stream)
        kms = []
        with ClockSampler(0) as clocks:
            for _ in range(args.steps):
                (dd, dr, rr), st = ctx.count_all(cd, cr, b, stream, stats=True)
                kms.append(st["kernel_ms"])
        assert int(dd.sum()) == nd * (nd - 1) // 2 and int(dr.sum()) == nd * nr and int(rr.sum()) == nr * (nr - 1) // 2
        g = np.random.default_rng(7)
        ds = w.data[np.sort(g.choice(nd, args.sub, replace=False))]
        rs = w.rand[np.sort(g.choice(nr, args.sub, replace=False))]
        sub = ctx.count_all(ctx.catalog3d(ds), ctx.catalog3d(rs), b)
    cores = os.cpu_count() or 1
    want = (oracle.count_auto(ds, w.edges, cores, euclid=True), oracle.count_cross(ds, rs, w.edges, cores, euclid=True),
            oracle.count_auto(rs, w.edges, cores, euclid=True))
    same = all(np.array_equal(a, c) for a, c in zip(sub, want))
    km = statistics.mean(kms)
    lane_ops = 6  # 3 FADD + 3 FFMA per pair on the FP32 pipe
    peak = 152 * 128 * 2.07e9
    print(json.dumps({
        "mode": "box3d", "metric": METRIC, "value": pairs / km * 1e3, "unit": UNIT, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": km, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"box: N_D={nd:,} clustered (4096 clusters sigma 2), N_R={nr:,} uniform, side 1000, "
                               "30 log distance bins 0.5-50, seed 0", "pairs_per_step": pairs},
        "roofline": {"bound": "alu", "lane_ops_per_pair": lane_ops,
                     "frac": pairs / (km / 1e3) * lane_ops / peak,
                     "peak": "152 SMs x 128 FP32 lanes x 2.07 GHz lane-ops/s (derived)"},
        "band": {"pairs": st["band_pairs"], "fraction": st["band_pairs"] / pairs},
        "subsample_parity": {"points_per_catalog": args.sub, "identical_to_oracle": same},
        "clocks": clocks.summary()}))
    assert same, "subsample histograms differ from the oracle"
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000, help="points per catalog")
    ap.add_argument("--cpu-sample", type=int, default=40_000,
                    help="points per catalog for the multi-threaded oracle timing and the subsample parity check")
    ap.add_argument("--cpu-sample-1t", type=int, default=10_000,
                    help="points per catalog for the single-threaded oracle timing (the cpu_baseline value)")
    ap.add_argument("--ref-sample", type=int, default=16_000, help="points per catalog per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-binary64 kernel comparison")
    ap.add_argument("--no-prune", action="store_true", help="skip the spatial-pruning launch of the default line")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact large / jackknife / serving records of the default line")
    ap.add_argument("--workload", default="octant_precision",
                    choices=["octant_precision", "jackknife", "serving", "large", "box3d"])
    ap.add_argument("--jobs", type=int, default=2000, help="serving: number of jobs")
    ap.add_argument("--workers", type=int, default=0, help="serving: job slots (0: the server's default, 32)")
    ap.add_argument("--sub", type=int, default=100_000, help="large: subsample points per catalog")
    ap.add_argument("--count-only", type=int, default=0, metavar="N",
                    help="profiling helper: one fused counting launch on the N-point octant workload")
    args = ap.parse_args()
    if args.count_only:
        return run_count_only(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "octant_precision":
        return {"jackknife": run_jackknife, "serving": run_serving, "large": run_large,
                "box3d": run_box3d}[args.workload](args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
