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
operations per pair (FMUL + 2 FFMA), counted as 6 flops, against the FP32
peak 152 SMs x 128 lanes x 2 flops x 2.07 GHz.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
FLOPS_PER_PAIR = 6            # 3 FP32 pipe lane-ops (FMUL + 2 FFMA), FMA convention
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.55: SMs x lanes x 2 x max SM clock
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
def oracle_sample(w, n_sample: int, threads: int):
    """Time the oracle on the first n_sample points of D and R (DD + DR + RR)."""
    import oracle
    d, r = w.data[:n_sample], w.rand[:n_sample]
    t0 = time.perf_counter()
    oracle.correlation(d, r, w.edges, threads=threads)
    dt = time.perf_counter() - t0
    pairs = n_sample * (n_sample - 1) + n_sample * n_sample
    return pairs / dt, dt, pairs


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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v, dt, sp = oracle_sample(w, args.cpu_sample, cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_sample:,} points of D and of R, DD+DR+RR = {sp:,} pairs, {dt:.1f} s"}

    kern_s = statistics.mean(kernel_ms) / 1e3
    achieved = st["pairs"] * FLOPS_PER_PAIR / kern_s / 1e12   # this rank's launch
    traffic = None
    prof = os.path.join(ROOT, "profiles", "count_kernel_traffic.json")
    if os.path.exists(prof):
        try:
            traffic = json.load(open(prof)).get("dram_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    cfg = workload_config(args.n, nbins)
    cfg["pairs_per_step"] = pairs
    cfg["parallelism"] = f"shards{world}" if world > 1 else "single"
    line = {
        "metric": METRIC, "value": pairs * args.steps / (elapsed_ms / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32", "precision": "FP32 screen + binary64 guard-band recheck, uint64 counts",
        "data": "synthetic", "config": cfg,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "count_kernel<512,8,screen> (fused DD/DR/RR)",
                     "kernel_ms": statistics.mean(kernel_ms),
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (no FP32 entry in "
                                    "MEASURED_PEAKS.json)"},
        "band": {"pairs": st["band_pairs"], "fraction": st["band_pairs"] / max(1, st["pairs"]),
                 "fp32_mismatch": st["band_mismatch"]},
        "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


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


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000, help="points per catalog")
    ap.add_argument("--cpu-sample", type=int, default=40_000, help="points per catalog for the oracle timing")
    ap.add_argument("--ref-sample", type=int, default=16_000, help="points per catalog per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count-only", type=int, default=0, metavar="N",
                    help="profiling helper: one fused counting launch on the N-point octant workload")
    args = ap.parse_args()
    if args.count_only:
        return run_count_only(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
