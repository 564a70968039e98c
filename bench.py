#!/usr/bin/env python3
"""Throughput of the Tucker/HOSVD of a Matern covariance tensor on GB300.

Workload (one step = one whole solve through the C-ABI): Matern nu = 1.2,
ell = 0.2, sigma2 = 1 on the 256^3 cell-centred grid in [-1, 1]^3, eps = 1e-6:
sample F, |F|^2, Gram of the unfoldings, leading eigenpairs and ranks, core
by chained TTMs, then the relative Frobenius error by direct subtraction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs independent
replicas of the solve (the path has no exchange step) and rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Matérn Tucker-HOSVD solves/s at rel err 1e-6 vs FP64 path; p50/p99 latency"
WORKLOAD = ("Matern nu=1.2 ell=0.2 sigma2=1, n=256^3 cell-centred grid on [-1,1]^3, eps=1e-6, "
            "rank cap 64; one solve (sample, Gram, eigenpairs, ranks, core, rel_error) per step")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "sliced"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                v = [t.strip() for t in line.split(",")]
                if len(v) >= 9:
                    rows.append(v)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(prob, seconds_cap=60.0):
    """The FP64 oracle, as it stands, on this host's cores: one whole solve."""
    import oracle
    from paper_1711_06874_gb300 import workloads

    oracle.build()
    k, g = workloads.oracle_kernel(prob, oracle), workloads.oracle_grid(prob, oracle)
    t = time.perf_counter()
    ref = oracle.hosvd(k, g, prob.eps, rmax=list(prob.rmax))
    dt = time.perf_counter() - t
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one whole FP64 oracle solve of the bench workload ({dt:.1f} s; ranks {ref['ranks']}, "
                      f"rel_error {ref['rel_error']:.3g})"}


def run_reference(args):
    """The oracle timed as the reference arm: each step one whole solve on the host cores."""
    rank, _, world = dist_info()
    if rank != 0:
        return 0
    import oracle
    from paper_1711_06874_gb300 import workloads

    oracle.build()
    prob = workloads.matern_n256(1e-6)
    k, g = workloads.oracle_kernel(prob, oracle), workloads.oracle_grid(prob, oracle)
    for _ in range(min(args.warmup, 1)):
        oracle.hosvd(k, g, prob.eps, rmax=list(prob.rmax))
    times = []
    budget = 240.0  # keep the whole arm within a few minutes
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t = time.perf_counter()
        ref = oracle.hosvd(k, g, prob.eps, rmax=list(prob.rmax))
        times.append(time.perf_counter() - t)
        if time.perf_counter() - t_all > budget:
            break
    total = sum(times)
    value = len(times) / total
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": len(times), "warmup": min(args.warmup, 1), "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)"},
        "rel_error": ref["rel_error"], "ranks": ref["ranks"],
        "latency_ms": {"p50": 1000 * statistics.median(times), "p99": 1000 * max(times)},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(times)} whole oracle solves of the bench workload"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_1711_06874_gb300 import binding, workloads

    rank, local_rank, world = dist_info()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    ctx = binding.Context(local_rank)
    prob = workloads.matern_n256(1e-6)
    prec_name = args.precision
    if prec_name == "auto":
        prec_name = "sliced" if getattr(binding, "SLICED_AVAILABLE", False) else "fp64"
    precision = binding.TK_SLICED_BF16 if prec_name == "sliced" else binding.TK_FP64
    stream = torch.cuda.Stream()

    def solve(p):
        res = ctx.tucker(prob, precision=p, stream=stream)
        err = res.rel_error(stream=stream)
        ranks = res.ranks
        res.free()
        return err, ranks

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(p, steps, warmup, profile=False):
        for _ in range(warmup):
            solve(p)
        if profile:
            ctx.profile(True)
        l0 = binding.Context.kernel_launches()
        barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0.record(stream)
        out = None
        for k in range(steps):
            ev[k][0].record(stream)
            out = solve(p)
            ev[k][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = binding.Context.kernel_launches() - l0
        ms = t0.elapsed_time(t1)
        lat = sorted(a.elapsed_time(b) for a, b in ev)
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile(False)
        if dist is not None:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, lat, launches, prof, out

    sampler = ClockSampler(local_rank)
    for _ in range(args.warmup):
        solve(precision)
    sampler.start()
    ms, lat, launches, prof, (err, (ranks, flags)) = timed(precision, args.steps, 0, profile=True)
    clocks = sampler.stop()
    value = args.steps * world / (ms / 1000.0)

    # the plain FP64 GPU path on the same workload (comparison of the metric)
    if precision != binding.TK_FP64:
        k64 = max(3, min(args.steps, 10))
        ms64, lat64, _, _, (err64, _) = timed(binding.TK_FP64, k64, 1)
        fp64 = {"value": k64 * world / (ms64 / 1000.0), "ms_per_step": ms64 / k64, "rel_error": err64}
    else:
        fp64 = {"value": value, "ms_per_step": ms / args.steps, "rel_error": err, "note": "this line is the FP64 path"}

    # end to end through the C-ABI with host buffers: parameters in, factors, core and error out
    import ctypes

    h2d = ctypes.sizeof(binding.Kernel) + ctypes.sizeof(binding.Grid) + ctypes.sizeof(binding.Opts)
    d2h = 0
    torch.cuda.synchronize()
    barrier()
    te = time.perf_counter()
    ke = args.steps
    for _ in range(ke):
        res = ctx.tucker(prob, precision=precision, stream=stream)
        e = res.rel_error(stream=stream)
        U = [res.factor(a) for a in range(3)]
        B = res.core()
        d2h = sum(u.nbytes for u in U) + B.nbytes + 8
        res.free()
    torch.cuda.synchronize()
    te = time.perf_counter() - te
    if dist is not None:
        t = torch.tensor([te], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        te = float(t.item())
    e2e = {"value": ke * world / te, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # roofline of the dominant stage (largest share of the profiled step)
    peaks, peak_src = load_peaks()
    stage_ms = {k: v[0] / max(1, args.steps) for k, v in prof.items()}
    n = prob.n[0]
    nmodes = 1  # isotropic shortcut: one Gram and one eigensolve per solve
    gram_launch_ms = prof["gram"][0] / max(1, prof["gram"][1])
    gram_flop = n * (n + 1) / 2 * n * n * 2.0  # unique entries of one G_k, K = n^2 products each
    if precision == binding.TK_FP64:
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        fp64_peak_tflops = 1.25 * sm_mhz / 2070.0  # nominal 1.25 TFLOP/s at 2070 MHz, scaled by the clock
        achieved = gram_flop / (gram_launch_ms * 1e-3) / 1e12
        roof = {"kernel": "k_gram_f64 (+ split-K reduce)", "bound": "alu", "achieved": achieved,
                "peak": fp64_peak_tflops, "unit": "TFLOP/s", "frac": achieved / fp64_peak_tflops,
                "traffic": None,
                "peak_source": "nominal FP64 1.25 TFLOP/s at 2070 MHz scaled to the sampled SM clock",
                "algorithmic_flop_per_launch": gram_flop}
    else:
        tc_peak = peaks["bf16_tflops_sustained"]
        achieved = gram_flop / (gram_launch_ms * 1e-3) / 1e12
        roof = {"kernel": "gram (sliced BF16)", "bound": "tensor", "achieved": achieved, "peak": tc_peak,
                "unit": "TFLOP/s", "frac": achieved / tc_peak, "traffic": None,
                "peak_source": f"bf16_tflops_sustained ({peak_src})", "algorithmic_flop_per_launch": gram_flop}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if precision == binding.TK_FP64 else "bf16-slices/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": prec_name, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: F (134 MB FP64) is resampled every step",
                   "isotropic_shortcut": True},
        "rel_error": err, "ranks": ranks, "flags": flags,
        "latency_ms": {"p50": statistics.median(lat), "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
        "fp64_path": fp64, "e2e": e2e, "gpu_launches": launches, "stages_ms_per_step": stage_ms,
        "roofline": roof, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
