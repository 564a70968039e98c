#!/usr/bin/env python3
"""Throughput of the Tucker/HOSVD of a Matern covariance tensor on GB300.

Default workload (one step = one whole solve through the C-ABI): Matern
nu = 1.2, ell = 0.2, sigma2 = 1 on the 256^3 cell-centred grid in [-1, 1]^3,
eps = 1e-6: sample F, Gram of the unfoldings, leading eigenpairs and ranks,
core by chained TTMs, then the relative Frobenius error by direct
subtraction.  --workload sweep: one step = the 256-instance n = 128 parameter
sweep in one tk_batch call.  --workload serving: the 2000-request Poisson
stream replayed in real time through the serving loop.  --workload spectral:
the default step on the Matern spectral density of Eq. (SD_matern), nu = 0.4,
alpha = 0.1 (FP64 Gram unless --precision says otherwise).  --workload als:
one Tucker-ALS sweep (Sec. 3.2) of the default workload's tensor, from its
HOSVD factors, through tk_als.  --workload multigrid: one multigrid Tucker
solve (Sec. 3.2) of the default workload, the HOSVD on the 64^3 grid and one
Tucker-ALS sweep on each of the 64^3, 128^3 and 256^3 grids, through
tk_multigrid.  --workload n512: the n = 512 solve (nu = 2.5, ell = 0.1), fused
sampling and slicing against the materialised octant tensor.  --workload
slater64: the n = 64 Slater solve (nu = 1/2, ell = 0.3, eps = 1e-8, FP64).
--workload c2t: canonical-to-Tucker (Sec. 3.4) of the sinc CP of 1/|x| on the
256^3 grid through tk_c2t.  --eps overrides the eps of the single-solve
workloads.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload single|sweep|serving|spectral|als|multigrid|n512|slater64|c2t] [--eps E]

Prints one JSON line.  Under torchrun (N > 1) every rank runs independent
replicas of the workload (the path has no exchange step) and rank 0 prints.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Matérn Tucker-HOSVD solves/s at rel err 1e-6 vs FP64 path; p50/p99 latency"
SPECTRAL_METRIC = "Matern spectral density (Eq. SD_matern) Tucker-HOSVD solves/s at rel err 1e-6; p50/p99 latency"
SPECTRAL_WORKLOAD = ("Matern spectral density nu=0.4 alpha=0.1 sigma2=1, n=256^3 cell-centred grid on [-1,1]^3, "
                     "eps=1e-6, rank cap 64; one solve (sample, Gram, eigenpairs, ranks, core, rel_error) per step")
WORKLOAD = ("Matern nu=1.2 ell=0.2 sigma2=1, n=256^3 cell-centred grid on [-1,1]^3, eps=1e-6, "
            "rank cap 64; one solve (sample, Gram, eigenpairs, ranks, core, rel_error) per step")
SWEEP = ("256 Matern instances, n=128^3 cell-centred grid on [-1,1]^3, nu~U[0.3,2.5], ell~logU[0.05,1], "
         "sigma2=1, eps=1e-6, rank cap 64, seeded PCG64(1711); one tk_batch call per step")
SERVING = ("2000 requests, Poisson arrivals 200/s, n uniform over {64,128,256,384}, nu~U[0.3,2.5], "
           "ell~logU[0.05,1], eps over {1e-4,1e-6,1e-8}, rank cap 64, seeded PCG64(6874); "
           "replayed in real time through the serving loop")
ALS_METRIC = "Tucker-ALS sweeps/s (modes 1, 2, 3 and the core) on the n=256 Matern tensor, FP64"
ALS_WORKLOAD = ("Matern nu=1.2 ell=0.2 sigma2=1, n=256^3 cell-centred grid on [-1,1]^3, F resident on the device; "
                "one tk_als sweep from the FP64 HOSVD's rank-11 factors (eps=1e-6) per step")
MG_METRIC = "Multigrid Tucker solves/s (HOSVD on 64^3, one ALS sweep per grid) on the n=256 Matern tensor, FP64"
MG_WORKLOAD = ("Matern nu=1.2 ell=0.2 sigma2=1, n=256^3 cell-centred grid on [-1,1]^3, eps=1e-6 ranks from the "
               "64^3 HOSVD, levels=2 (64 -> 128 -> 256), 1 sweep per grid, F sampled on the device per grid")
MG_LEVELS, MG_SWEEPS = 2, 1
N512_METRIC = "Matern Tucker-HOSVD solves/s, n=512 (nu=2.5, ell=0.1, eps=1e-6); p50/p99 latency"
N512_WORKLOAD = ("Matern nu=2.5 ell=0.1 sigma2=1, n=512^3 cell-centred grid on [-1,1]^3, eps={eps:g}, rank cap 64; "
                 "one solve (sample, Gram, eigenpairs, ranks, core, rel_error) per step")
C1_METRIC = "Slater (Matern nu=1/2) Tucker-HOSVD solves/s, n=64, eps=1e-8, FP64; p50/p99 latency"
C1_WORKLOAD = ("Matern nu=0.5 (Slater) ell=0.3 sigma2=1, n=64^3 cell-centred grid on [-1,1]^3, eps={eps:g}, "
               "rank cap 20; one solve (sample, Gram, eigenpairs, ranks, core, rel_error) per step")
C2T_METRIC = "Canonical-to-Tucker (Sec. 3.4) solves/s: RHOSVD + 1 ALS sweep of the sinc CP of 1/|x|, FP64"
C2T_WORKLOAD = ("sinc CP of the Newton kernel 1/|x| (M=64, R=129 terms, h_M = 3 log(M)/M), collocated on the "
                "256^3 cell-centred grid on [-1,1]^3, eps=1e-6, one tk_c2t call (RHOSVD and 1 sweep) per step, "
                "CP input resident on the device")
FP64_TFLOPS_NOMINAL = 1.25  # GB300 FP64 at 2070 MHz (nominal; the pipe the eigensolver and TTMs run on)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "sliced", "bf16x3", "tf32x3"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="default K splits (for profiling runs)")
    p.add_argument("--workload", default="single", choices=["single", "sweep", "serving", "spectral", "als",
                                                                       "multigrid", "n512", "slater64", "c2t"])
    p.add_argument("--eps", type=float, default=None, help="eps of the single-solve workloads (default: theirs)")
    return p.parse_args()


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized():
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units of all ranks (independent replicas) per second of the slowest rank."""
    return units_per_rank * world / seconds


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


def _dtype(binding, precision):
    return {binding.TK_FP64: "f64", binding.TK_SLICED_BF16: "bf16-slices/f64", binding.TK_BF16X3: "bf16x3/f32",
            binding.TK_TF32X3: "tf32x3/f32"}[precision]


def _flush_l2(torch, buf, stream):
    with torch.cuda.stream(stream):
        buf.add_(1.0)


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


JACOBI_SWEEPS = 3  # rotation sweeps on the n = 256 workload's Rayleigh-Ritz matrix (device counter)


def _knu_flops(prob):
    """FP64 operations of the K_nu table of the cubic isotropic workload: per
    distinct s, the Miller recurrence (5 per step, N = 12 + ceil(180/x) steps)
    or Temme's series (about 14 per term, 20 terms) plus about 80 for the
    prefactor and the forward recurrence."""
    n = prob.n[0]
    hstep = prob.b[0] / n
    nu, ell = prob.nu, prob.ell[0]
    Q = (3 * (n - 1) ** 2 - 3) // 8 + 1 if n % 2 == 0 else 3 * ((n - 1) // 2) ** 2 + 1
    tot = 0.0
    for q in range(Q):
        s = 8 * q + 3 if n % 2 == 0 else 4 * q
        x = math.sqrt(2 * nu) * hstep * math.sqrt(s) / ell
        tot += 80 + (14 * 20 if x <= 1.5 else 5 * (12 + math.ceil(180.0 / x)))
    return tot


def _gram_tc_issued(h):
    """BF16 flops the tensor-core Gram issues for one h x h octant Gram: 21
    slice pairs on every 128 x 64 block touching the upper triangle."""
    nrt, nct = (h + 127) // 128, (h + 63) // 64
    nb = sum(max(0, nct - (i * 128) // 64) for i in range(nrt))
    return 21 * 2.0 * 128 * 64 * (h * h) * nb


def _roofline(prof, prob, precision, clocks, peaks, peak_src, instances=1):
    """Roofline of the kernel with the largest time per step among the ones
    the library times on their own (nested stage events on the solve stream):
    the K_nu table, the tensor-core Gram, the eigensolver's QR and Jacobi.
    Every fraction is against the whole GPU's peak of the pipe the kernel is
    bound by; `instances` problems of the same shape share each launch."""
    n = prob.n[0]
    h = (n + 1) // 2
    ms = min(h, 12 + 4)  # subspace of the first eigenpair pass (12 pairs, 4 extra columns)
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_gpu = FP64_TFLOPS_NOMINAL * sm_mhz / 2070.0
    fp64_src = ("GPU FP64: nominal 1.25 TFLOP/s at 2070 MHz (152 SMs x 2 FMA/clk x 2 flop; an FMA-chain probe "
                "measured 1.19), scaled to the sampled SM clock")
    have = {k: prof[k] for k in ("table", "gram_tc", "qr", "jacobi") if k in prof and prof[k][1] > 0}
    if not have:
        return {"kernel": None, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}
    top = max(have, key=lambda k: have[k][0])
    t = have[top][0] / have[top][1] * 1e-3  # s per launch
    if instances > 1 and top in ("qr", "jacobi"):
        # instances needing more pairs run the stage again on a subset: take the
        # whole step's stage time against the first pass's work (a lower bound)
        t = have[top][0] * 1e-3
    out = {"kernel": None, "stage_ms_per_launch": t * 1e3, "traffic": None, "instances_per_launch": instances}
    if top == "gram_tc":
        issued = _gram_tc_issued(h) * instances
        ach = issued / t / 1e12
        pk = peaks["bf16_tflops_sustained"]
        out.update(kernel="k_gram_tc (sliced BF16 Gram)", bound="tensor", achieved=ach, peak=pk, unit="TFLOP/s",
                   frac=ach / pk, peak_source=f"bf16_tflops_sustained ({peak_src}), issued slice products",
                   algorithmic_flop_per_launch=issued)
    elif top in ("qr", "jacobi"):
        if top == "qr":
            work = 8.0 * h * ms * ms - 8.0 * ms ** 3 / 3.0  # Householder QR plus the explicit Q
            name = "k_qr_factor64 + k_form_q (FP64 Householder QR of the subspace block)"
        else:
            work = 7.0 * ms ** 3 * JACOBI_SWEEPS  # 7 m^3 flops per sweep (A two-sided, V one-sided)
            name = "k_jacobi_strided (FP64 Jacobi of the Rayleigh-Ritz matrix)"
        work *= instances
        ach = work / t / 1e12
        out.update(kernel=name, bound="alu", achieved=ach, peak=fp64_gpu, unit="TFLOP/s", frac=ach / fp64_gpu,
                   frac_of_the_sms_used=ach / (fp64_gpu * min(152, instances) / 152.0),
                   peak_source=fp64_src + "; frac_of_the_sms_used: against the FP64 of the SMs the launch occupies "
                                          "(one CTA per instance), a diagnosis only",
                   algorithmic_flop_per_launch=work)
    else:
        work = _knu_flops(prob) * instances
        ach = work / t / 1e12
        out.update(kernel="k_table_b (K_nu per distinct s, FP64)", bound="alu", achieved=ach, peak=fp64_gpu,
                   unit="TFLOP/s", frac=ach / fp64_gpu, peak_source=fp64_src, algorithmic_flop_per_launch=work)
    out["per_step_ms"] = {k: v[0] for k, v in have.items()}
    if "gram_tc" in have and top != "gram_tc":
        tg = have["gram_tc"][0] / have["gram_tc"][1] * 1e-3
        issued = _gram_tc_issued(h) * instances
        out["gram_tc"] = {"achieved": issued / tg / 1e12, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                          "frac": issued / tg / 1e12 / peaks["bf16_tflops_sustained"],
                          "ms_per_launch": tg * 1e3, "algorithmic_flop_per_launch": issued}
    return out


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
    prec_name = args.precision
    if prec_name == "auto" and args.workload == "slater64":
        prec_name = "fp64"  # the FP64 configuration of the small Slater case
    if prec_name == "auto" and args.workload == "spectral":
        # the sliced Gram flags eps = 1e-6 as below its accuracy on this sharply
        # peaked function and its E lands above 1e-6: the FP64 Gram meets it
        prec_name = "fp64"
    if prec_name == "auto":
        prec_name = "sliced" if getattr(binding, "SLICED_AVAILABLE", False) else "fp64"
    precision = {"sliced": binding.TK_SLICED_BF16, "bf16x3": binding.TK_BF16X3, "tf32x3": binding.TK_TF32X3,
                 "fp64": binding.TK_FP64}[prec_name]
    stream = torch.cuda.Stream()
    # written between timed steps so that no step starts with a warm L2 (129 MB)
    flush = torch.zeros(64 << 20, dtype=torch.float64, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    def allmax(x):
        return max_over_ranks(x, dist, "cuda")

    def timed(step, steps, warmup, profile=False, cleanup=None):
        """Per-step CUDA events on the solve stream; L2 flushed between steps.
        cleanup(out) runs after a step's closing event (host bookkeeping such
        as freeing results, outside the step)."""
        for _ in range(warmup):
            out = step()
            if cleanup:
                cleanup(out)
        if profile:
            ctx.profile(True)
        l0 = binding.Context.kernel_launches()
        barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        out = None
        for k in range(steps):
            _flush_l2(torch, flush, stream)
            ev[k][0].record(stream)
            out = step()
            ev[k][1].record(stream)
            if cleanup:
                out = cleanup(out)
        torch.cuda.synchronize()
        barrier()
        launches = binding.Context.kernel_launches() - l0
        lat = [a.elapsed_time(b) for a, b in ev]
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile(False)
        return allmax(sum(lat)), lat, launches, prof, out

    peaks, peak_src = load_peaks()
    # the sliced Gram's K split picked by timing (its result does not depend on
    # it); not while serving, where every new batch size would pause to time
    tune_path = os.path.join(tempfile.gettempdir(), f"tk_tune_{os.getpid()}.json")
    tuning = args.workload != "serving" and not args.no_tune
    if tuning:
        ctx.tune(True, tune_path)
    if args.workload in ("single", "spectral", "n512", "slater64"):
        line = bench_single(args, torch, binding, workloads, ctx, precision, prec_name, stream, timed, barrier,
                            allmax, world, peaks, peak_src)
    elif args.workload == "c2t":
        line = bench_c2t(args, torch, binding, ctx, stream, timed, barrier, allmax, world, peaks)
    elif args.workload == "multigrid":
        line = bench_multigrid(args, torch, binding, workloads, ctx, stream, timed, barrier, allmax, world, peaks)
    elif args.workload == "als":
        line = bench_als(args, torch, binding, workloads, ctx, stream, timed, barrier, allmax, world, peaks)
    elif args.workload == "sweep":
        line = bench_sweep(args, torch, binding, workloads, ctx, precision, prec_name, stream, timed, world, peaks,
                           peak_src)
    else:
        line = bench_serving(args, torch, binding, workloads, ctx, precision, prec_name, world, allmax, peaks,
                             peak_src)
    chosen = {}
    if os.path.exists(tune_path):
        with open(tune_path) as fh:
            chosen = json.load(fh)
        os.unlink(tune_path)
    line.setdefault("config", {})["autotune"] = {
        "what": "K split of the sliced tensor-core Gram chosen by timing (the Gram does not depend on it)",
        "chunks_of_256_per_cta": chosen} if tuning else "off (default splits)"
    ctx.tune(False, "")
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def bench_single(args, torch, binding, workloads, ctx, precision, prec_name, stream, timed, barrier, allmax, world,
                 peaks, peak_src):
    rank, local_rank, _ = dist_info()
    spectral = args.workload == "spectral"
    wk = args.workload
    # the spectral density workload: the paper's nu = 0.4 with its smaller alpha
    if spectral:
        prob = workloads.problem(workloads.MATERN_SD, nu=0.4, p=0.1, n=256, eps=args.eps or 1e-6, rmax=64)
        metric, workload = SPECTRAL_METRIC, SPECTRAL_WORKLOAD
    elif wk == "n512":
        prob = workloads.matern_n512(args.eps or 1e-6)
        metric, workload = N512_METRIC, N512_WORKLOAD.format(eps=prob.eps)
    elif wk == "slater64":
        prob = workloads.slater_n64(args.eps or 1e-8)
        metric, workload = C1_METRIC, C1_WORKLOAD.format(eps=prob.eps)
    else:
        prob = workloads.matern_n256(args.eps or 1e-6)
        metric, workload = METRIC, WORKLOAD.replace("eps=1e-6", f"eps={prob.eps:g}")

    def solve(p, fused=True):
        # E from a second, independent sampling of F that the library runs on a
        # side stream while the eigenpairs are computed
        res = ctx.tucker(prob, precision=p, with_error=True, stream=stream, fused_eval=fused)
        err = res.solve_error
        ranks = res.ranks
        res.free()
        return err, ranks

    sampler = ClockSampler(local_rank)
    for _ in range(args.warmup):
        solve(precision)
    sampler.start()
    ms, lat, launches, _, (err, (ranks, flags)) = timed(lambda: solve(precision), args.steps, 0)
    clocks = sampler.stop()
    value = whole_job_rate(args.steps, world, ms / 1000.0)
    # per-stage device times from a separate pass with the library's stage
    # events on (they add work to the stream, so not in the timed steps)
    kprof = max(3, min(args.steps, 10))
    _, _, _, prof, _ = timed(lambda: solve(precision), kprof, 0, profile=True)

    # the plain FP64 GPU path on the same workload (comparison of the metric)
    if precision != binding.TK_FP64:
        k64 = max(3, min(args.steps, 10))
        ms64, lat64, _, _, (err64, _) = timed(lambda: solve(binding.TK_FP64), k64, 1)
        fp64 = {"value": k64 * world / (ms64 / 1000.0), "ms_per_step": ms64 / k64, "rel_error": err64}
    else:
        fp64 = {"value": value, "ms_per_step": ms / args.steps, "rel_error": err, "note": "this line is the FP64 path"}

    # n = 512: the sampling and slicing fused (the default) against the octant
    # tensor materialised first, the same solve otherwise
    materialised = None
    if wk == "n512" and precision == binding.TK_SLICED_BF16:
        kmt = max(3, min(args.steps, 10))
        msm, latm, _, _, (errm, _) = timed(lambda: solve(precision, fused=False), kmt, 1)
        materialised = {"value": kmt * world / (msm / 1000.0), "ms_per_step": msm / kmt, "rel_error": errm,
                        "latency_ms": {"p50": statistics.median(latm), "p99": _pct(latm, 0.99)},
                        "note": "fused_eval=0: FP64 octant tensor sampled into HBM, then sliced"}
    # the two FP32-class split variants on the same workload: reported with
    # their measured E, outside the metric when E misses eps
    variants = {}
    if not spectral and wk != "slater64":
        for vname, vp in (("bf16x3", binding.TK_BF16X3), ("tf32x3", binding.TK_TF32X3)):
            if vp == precision:
                continue
            kv = max(3, min(args.steps, 10))
            msv, _, _, _, (errv, (rv, fv)) = timed(lambda: solve(vp), kv, 1)
            variants[vname] = {"value": kv * world / (msv / 1000.0), "ms_per_step": msv / kv, "rel_error": errv,
                               "ranks": rv, "flags": fv, "meets_eps": errv <= prob.eps,
                               "within_2x_fp64_path_E": errv <= 2 * fp64["rel_error"]}
        variants["note"] = ("Gram from a two-term split with FP32 sums (tcgen05 kind::f16 / kind::tf32); a variant "
                            "whose E misses eps is outside the metric")

    # end to end through the C-ABI with host buffers: parameters in, factors, core and error out
    import ctypes

    h2d = ctypes.sizeof(binding.Kernel) + ctypes.sizeof(binding.Grid) + ctypes.sizeof(binding.Opts)
    d2h = 0
    torch.cuda.synchronize()
    barrier()
    te = time.perf_counter()
    ke = args.steps
    for _ in range(ke):
        res = ctx.tucker(prob, precision=precision, with_error=True, stream=stream)
        e = res.solve_error
        *U, B = res.factors_and_core(stream=stream)
        d2h = sum(u.nbytes for u in U) + B.nbytes + 8
        res.free()
    torch.cuda.synchronize()
    te = allmax(time.perf_counter() - te)
    e2e = {"value": ke * world / te, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    stage_ms = {k: v[0] / kprof for k, v in prof.items()}
    per_step = {k: (v[0] / kprof, v[1] / kprof) for k, v in prof.items()}
    if spectral:
        # the roofline formulas below model the Matern workload's first pass
        # (K_nu table, 16-column subspace); this workload escalates its ranks
        roof = {"kernel": None, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "note": "reported for the default workload only"}
    else:
        roof = _roofline(per_step, prob, precision, clocks, peaks, peak_src)
    line = {
        "metric": metric, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": _dtype(binding, precision),
        "data": "synthetic",
        "config": {"workload": workload, "precision": prec_name,
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (512 MB written on the solve stream, outside the step events)",
                   "isotropic_shortcut": True, "reflect_fold": True},
        "rel_error": err, "ranks": ranks, "flags": flags,
        "latency_ms": {"p50": statistics.median(lat), "p99": _pct(lat, 0.99)},
        "fp64_path": fp64, "precision_variants": variants, "materialised": materialised, "e2e": e2e,
        "gpu_launches": launches,
        "stages_ms_per_step": stage_ms,
        "roofline": roof, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if wk == "n512":
            # the whole oracle solve at n = 512 takes minutes: the same problem at
            # n = 256, scaled by (512 / 256)^4, the growth of its Gram
            small = workloads.problem(prob.kind, nu=prob.nu, ell=prob.ell[0], n=256, eps=prob.eps, rmax=64)
            cb = cpu_baseline(small)
            cb["value"] /= 16.0
            cb["sample"] = ("extrapolated: " + cb["sample"].replace("bench workload", "n=256 solve of the same "
                            "parameters") + ", rate divided by (512/256)^4 = 16 (the Gram's n^4 cost)")
            line["cpu_baseline"] = cb
        else:
            line["cpu_baseline"] = cpu_baseline(prob)
    return line


def _c2t_flops(n, R, r, sweeps):
    """Algorithmic FP64 work of one tk_c2t call: the side matrices' Grams for
    |A|^2 (R x R) and for the RHOSVD (n x n), then per sweep and mode the
    single-hole unfolding M (n x r_m r_q), its Gram and W = Z^T U; the core."""
    f = sum(2.0 * n[l] * R * R + 2.0 * n[l] * n[l] * R + 2.0 * r[l] * n[l] * R for l in range(3))
    for _ in range(sweeps):
        for l in range(3):
            m, q = [a for a in range(3) if a != l]
            rmq = r[m] * r[q]
            f += 2.0 * n[l] * R * rmq + 2.0 * n[l] * n[l] * rmq + 2.0 * r[l] * n[l] * R + 2.0 * rmq * R
    return f + 2.0 * R * r[0] * r[1] * r[2]


def bench_c2t(args, torch, binding, ctx, stream, timed, barrier, allmax, world, peaks):
    rank, local_rank, _ = dist_info()
    from paper_1711_06874_gb300 import cp_inputs

    n, M, eps, sweeps = 256, 64, args.eps or 1e-6, 1
    c, U = cp_inputs.newton_sinc_cp(n, M)
    R = c.size
    cd = torch.from_numpy(c).cuda()
    Ud = [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in U]

    def step():
        res, hist = ctx.c2t(cd, Ud, eps, sweeps, stream=stream)
        return res

    def done(res):
        r = res.ranks[0]
        res.free()
        return r

    sampler = ClockSampler(local_rank)
    for _ in range(args.warmup):
        done(step())
    sampler.start()
    ms, lat, launches, _, ranks = timed(step, args.steps, 0, cleanup=done)
    clocks = sampler.stop()
    value = whole_job_rate(args.steps, world, ms / 1000.0)
    ranks = list(ranks)
    # end to end: the CP input in from pinned host memory, factors and core out
    ch = torch.from_numpy(c).pin_memory()
    Uh = [torch.from_numpy(np.ascontiguousarray(u)).pin_memory() for u in U]
    h2d = ch.numel() * 8 + sum(u.numel() * 8 for u in Uh)
    d2h = 8 * (ranks[0] * ranks[1] * ranks[2] + sum(n * r for r in ranks))
    torch.cuda.synchronize()
    barrier()
    te = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            cd.copy_(ch, non_blocking=True)
            for a in range(3):
                Ud[a].copy_(Uh[a], non_blocking=True)
        res, _ = ctx.c2t(cd, Ud, eps, sweeps, stream=stream)
        res.factors_and_core(stream=stream)
        res.free()
    te = allmax(time.perf_counter() - te)
    e2e = {"value": args.steps * world / te, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    flop = _c2t_flops((n, n, n), R, ranks, sweeps)
    step_ms = ms / args.steps
    sm = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = FP64_TFLOPS_NOMINAL * sm / 2070.0
    achieved = flop / (step_ms * 1e-3) / 1e12
    roof = {"kernel": "tk_c2t (whole call: FP64 Grams, single-hole unfoldings, subspace eigensolves)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "algorithmic_flop_per_launch": flop,
            "peak_source": "GPU FP64: nominal 1.25 TFLOP/s at 2070 MHz, scaled to the sampled SM clock"}
    line = {
        "metric": C2T_METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": C2T_WORKLOAD.replace("eps=1e-6", f"eps={eps:g}"), "precision": "fp64",
                   "parallelism": f"replicas x{world}", "l2": "CP input 0.8 MB resident; no flush", "ranks": ranks},
        "latency_ms": {"p50": statistics.median(lat), "p99": _pct(lat, 0.99)},
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t = time.perf_counter()
        oracle.c2t(c, U, eps, sweeps)
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "solves/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"one whole oracle c2t of the bench input ({dt:.2f} s, "
                                                            f"LAPACK SVDs through numpy)"}
    return line


def _als_flops(n, r):
    """Algorithmic FP64 work of one sweep: the two contractions over F
    (F x_3 U3^T serves modes 1 and 2, F x_1 U1^T mode 3), the second
    products, the three Grams of the single-hole unfoldings and the core."""
    n1, n2, n3 = n
    r1, r2, r3 = r
    big = 2.0 * n1 * n2 * n3 * (r3 + r1)
    small = 2.0 * (n1 * n2 * r2 * r3 + r1 * n1 * n2 * r3 + r1 * r2 * n2 * n3)
    grams = 2.0 * (n1 * n1 * r2 * r3 + n2 * n2 * r1 * r3 + n3 * n3 * r1 * r2)
    return big + small + grams + 2.0 * r1 * r2 * r3 * n3


def bench_als(args, torch, binding, workloads, ctx, stream, timed, barrier, allmax, world, peaks):
    rank, local_rank, _ = dist_info()
    prob = workloads.matern_n256(1e-6)
    res = ctx.tucker(prob, precision=binding.TK_FP64)
    ranks, _ = res.ranks
    U0h = [res.factor(a) for a in range(3)]
    hosvd_core2 = float((res.core() ** 2).sum())
    res.free()
    n = tuple(prob.n)
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.eval(prob, F)
    U0 = [torch.from_numpy(u).cuda() for u in U0h]
    U = [u.clone() for u in U0]
    B = torch.empty(ranks, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    def step():
        with torch.cuda.stream(stream):
            for a in range(3):
                U[a].copy_(U0[a])
        return ctx.als(F, U, B, 1, stream=stream)

    sampler = ClockSampler(local_rank)
    for _ in range(args.warmup):
        step()
    sampler.start()
    ms, lat, launches, _, hist = timed(step, args.steps, 0)
    clocks = sampler.stop()
    value = whole_job_rate(args.steps, world, ms / 1000.0)

    # end to end with host buffers: F and the starting factors in, factors and core out
    Fh = F.cpu().pin_memory()
    Uh = [u.pin_memory() for u in (torch.from_numpy(x) for x in U0h)]
    Bh = torch.empty(ranks, dtype=torch.float64).pin_memory()
    Uo = [torch.empty_like(u).pin_memory() for u in Uh]
    h2d = Fh.numel() * 8 + sum(u.numel() * 8 for u in Uh)
    d2h = Bh.numel() * 8 + sum(u.numel() * 8 for u in Uo)
    torch.cuda.synchronize()
    barrier()
    te = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            F.copy_(Fh, non_blocking=True)
            for a in range(3):
                U[a].copy_(Uh[a], non_blocking=True)
        ctx.als(F, U, B, 1, stream=stream)
        with torch.cuda.stream(stream):
            for a in range(3):
                Uo[a].copy_(U[a], non_blocking=True)
            Bh.copy_(B, non_blocking=True)
        stream.synchronize()
    te = allmax(time.perf_counter() - te)
    e2e = {"value": args.steps * world / te, "unit": "sweeps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    flop = _als_flops(n, ranks)
    step_ms = ms / args.steps
    sm = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = FP64_TFLOPS_NOMINAL * sm / 2070.0
    achieved = flop / (step_ms * 1e-3) / 1e12
    roof = {"kernel": "tk_als sweep (whole call: two FP64 contractions over F, three eigensolves)", "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "peak_source": "GPU FP64: nominal 1.25 TFLOP/s at 2070 MHz, scaled to the sampled SM clock",
            "algorithmic_flop_per_launch": flop}
    line = {
        "metric": ALS_METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": ALS_WORKLOAD, "precision": "fp64", "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (512 MB written on the solve stream, outside the step events)",
                   "ranks": ranks},
        "core_norm2": {"hosvd": hosvd_core2, "after_sweep": [float(x) for x in hist]},
        "latency_ms": {"p50": statistics.median(lat), "p99": _pct(lat, 0.99)},
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        Fo = oracle.tensor(workloads.oracle_kernel(prob, oracle), workloads.oracle_grid(prob, oracle))
        t = time.perf_counter()
        oracle.hooi(Fo, U0h, 1)
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "sweeps/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"one whole oracle sweep of the bench tensor ({dt:.1f} s)"}
    return line


def bench_multigrid(args, torch, binding, workloads, ctx, stream, timed, barrier, allmax, world, peaks):
    rank, local_rank, _ = dist_info()
    prob = workloads.matern_n256(1e-6)

    def step():
        return ctx.multigrid(prob, MG_LEVELS, MG_SWEEPS, precision=binding.TK_FP64, stream=stream)

    def done(res):
        ranks = res.ranks[0]
        res.free()
        return ranks

    sampler = ClockSampler(local_rank)
    for _ in range(args.warmup):
        done(step())
    sampler.start()
    ms, lat, launches, _, ranks = timed(step, args.steps, 0, cleanup=done)
    clocks = sampler.stop()
    value = whole_job_rate(args.steps, world, ms / 1000.0)
    ranks = list(ranks)

    # end to end: the request in, the factors and core out to host memory
    d2h = 8 * (ranks[0] * ranks[1] * ranks[2] + sum(prob.n[a] * ranks[a] for a in range(3)))
    torch.cuda.synchronize()
    barrier()
    te = time.perf_counter()
    for _ in range(args.steps):
        res = step()
        res.factors_and_core(stream=stream)
        res.free()
    te = allmax(time.perf_counter() - te)
    e2e = {"value": args.steps * world / te, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h}

    # algorithmic FP64 work: one ALS sweep per grid (the 64^3 HOSVD is small next to it)
    n = tuple(prob.n)
    flop = sum(_als_flops(tuple(v >> (MG_LEVELS - lv) for v in n), ranks) for lv in range(MG_LEVELS + 1))
    step_ms = ms / args.steps
    sm = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = FP64_TFLOPS_NOMINAL * sm / 2070.0
    achieved = flop / (step_ms * 1e-3) / 1e12
    roof = {"kernel": "tk_multigrid (whole call: ALS contractions over F on three grids, K_nu sampling, HOSVD "
                      "on 64^3)", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "GPU FP64: nominal 1.25 TFLOP/s at 2070 MHz, scaled to the sampled SM clock",
            "algorithmic_flop_per_launch": flop}
    line = {
        "metric": MG_METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": MG_WORKLOAD, "precision": "fp64", "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (512 MB written on the solve stream, outside the step events)",
                   "ranks": ranks},
        "latency_ms": {"p50": statistics.median(lat), "p99": _pct(lat, 0.99)},
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t = time.perf_counter()
        oracle.multigrid(workloads.oracle_kernel(prob, oracle), workloads.oracle_grid(prob, oracle), prob.eps,
                         MG_LEVELS, MG_SWEEPS, rmax=list(prob.rmax))
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "solves/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"one whole oracle multigrid solve of the bench workload "
                                                            f"({dt:.1f} s)"}
    return line


def bench_sweep(args, torch, binding, workloads, ctx, precision, prec_name, stream, timed, world, peaks, peak_src):
    rank, local_rank, _ = dist_info()
    probs = workloads.sweep()

    # the C structs of the 256 requests are marshalled once, like inputs already resident
    bargs = {p: binding.BatchArgs(probs, precision=p) for p in {precision, binding.TK_FP64}}

    def step(p=precision):
        return ctx.batch(bargs[p], stream=stream)

    def cleanup(rs):
        ranks = [r.ranks[0][0] for r in rs]
        for r in rs:
            r.free()
        return ranks

    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, lat, launches, _, ranks = timed(step, args.steps, args.warmup, cleanup=cleanup)
    clocks = sampler.stop()
    value = len(probs) * args.steps * world / (ms / 1000.0)
    # per-stage device times from a separate pass with the library's stage events on
    kprof = max(2, min(args.steps, 3))
    _, _, _, prof, _ = timed(step, kprof, 0, profile=True, cleanup=cleanup)
    # accuracy of every instance, outside the timed region
    rs = ctx.batch(probs, precision=precision, stream=stream)
    errs = [r.rel_error(stream=stream) for r in rs]
    flags = [r.ranks[1][0] for r in rs]
    for r in rs:
        r.free()
    ok = sum(1 for e, p, f in zip(errs, probs, flags) if e <= p.eps * (1 + 1e-6) or (f & binding.TK_RANK_CAPPED))
    fp64 = None
    if precision != binding.TK_FP64:
        k64 = max(2, min(args.steps, 3))
        ms64, _, _, _, _ = timed(lambda: step(binding.TK_FP64), k64, 1, cleanup=cleanup)
        fp64 = {"value": len(probs) * k64 * world / (ms64 / 1000.0), "ms_per_step": ms64 / k64}
    line = {
        "metric": "Matern Tucker-HOSVD solves/s, 256-instance n=128 sweep (tk_batch)", "value": value,
        "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype(binding, precision), "data": "synthetic",
        "config": {"workload": SWEEP, "precision": prec_name, "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps; the batch's octant tensors (537 MB) exceed L2"},
        "latency_ms": {"p50": statistics.median(lat), "p99": _pct(lat, 0.99)},
        "ranks": {"min": min(ranks), "max": max(ranks), "mean": sum(ranks) / len(ranks)},
        "rel_error": {"max": max(errs), "within_eps_or_capped": ok, "count": len(errs)},
        "fp64_path": fp64, "gpu_launches": launches,
        "stages_ms_per_step": {k: v[0] / kprof for k, v in prof.items()},
        "roofline": _roofline({k: (v[0] / kprof, v[1] / kprof) for k, v in prof.items()},
                              probs[0], precision, clocks, peaks, peak_src, instances=len(probs)),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t = time.perf_counter()
        for p in probs[:2]:
            oracle.hosvd(workloads.oracle_kernel(p, oracle), workloads.oracle_grid(p, oracle), p.eps,
                         rmax=list(p.rmax))
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": 2 / dt, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": f"first 2 of the 256 sweep instances, whole FP64 oracle solves "
                                          f"({dt:.1f} s), extrapolated per solve"}
    return line


def bench_serving(args, torch, binding, workloads, ctx, precision, prec_name, world, allmax, peaks, peak_src):
    rank, local_rank, _ = dist_info()
    stream = workloads.serving_stream()

    def replay(p, reqs, realtime=True):
        """Submits the requests at their arrival times (realtime) or all at once
        (saturated: the queue never runs dry); throughput = requests / time from
        the first submission to the end of the last request's batch."""
        ctx.serve_start(workers=2)
        t0 = time.perf_counter()
        tickets = []
        for at, q in reqs:
            if realtime:
                d = at - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
            tickets.append((time.perf_counter() - t0, ctx.submit(q, precision=p)))
        lats, ends = [], []
        for ts, t in tickets:
            res, lat = ctx.poll(t, wait_s=600.0)
            res.free()
            lats.append(lat)
            ends.append(ts + lat)
        stats = ctx.serve_stats()
        ctx.serve_stop()
        span = max(ends)
        return len(reqs) / span, lats, stats

    def summary(v, lats, stats):
        lm = [1000 * x for x in lats]
        return {"value": v * world, "latency_ms": {"p50": statistics.median(lm), "p99": _pct(lm, 0.99),
                                                   "max": max(lm)}, "batches": stats["batches"],
                "max_batch_seen": stats["max_batch_seen"]}

    # warm-up: a few requests of every size
    warm = [(0.0, workloads.problem(0, nu=1.0, ell=0.3, n=n, eps=1e-6, rmax=64)) for n in (64, 128, 256, 384)]
    replay(precision, warm)
    sampler = ClockSampler(local_rank)
    sampler.start()
    value, lats, stats = replay(precision, stream)
    sat = {prec_name: summary(*replay(precision, stream, realtime=False))}
    clocks = sampler.stop()
    fp64 = None
    if precision != binding.TK_FP64:
        replay(binding.TK_FP64, warm)
        v64, l64, s64 = replay(binding.TK_FP64, stream)
        fp64 = {"value": v64, "latency_ms": {"p50": 1000 * statistics.median(l64), "p99": 1000 * _pct(l64, 0.99)},
                "batches": s64["batches"]}
        sat["fp64"] = summary(*replay(binding.TK_FP64, stream, realtime=False))
        sat["speedup_over_fp64"] = sat[prec_name]["value"] / sat["fp64"]["value"]
    sat["note"] = ("the same 2000 requests submitted all at once (closed queue, above capacity): solves/s from the "
                   "first submission to the last result, latency from submission to the end of the request's batch")
    # the stream's costliest requests (n = 384) as one profiled tk_batch: the
    # serving path's dominant kernel and its roofline
    big = [q for _, q in stream if q.n[0] == 384][:16]
    ctx.profile(True)
    for r in ctx.batch(big, precision=precision):
        r.free()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    roof = _roofline(prof, big[0], precision, clocks, peaks, peak_src, instances=len(big))
    roof["sample"] = f"one profiled tk_batch of the stream's first {len(big)} n=384 requests"
    lat_ms = [1000 * x for x in lats]
    return {
        "metric": "Matern Tucker-HOSVD serving solves/s with p50/p99 latency", "value": value * world,
        "unit": "solves/s", "n_gpus": world, "steps": len(stream), "warmup": len(warm),
        "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype(binding, precision), "data": "synthetic",
        "config": {"workload": SERVING, "precision": prec_name, "workers": 2,
                   "l2": "requests of up to 24 MB octant tensors stream through; no flush"},
        "latency_ms": {"p50": statistics.median(lat_ms), "p99": _pct(lat_ms, 0.99), "max": max(lat_ms)},
        "serve_stats": stats, "fp64_path": fp64, "saturated": sat, "roofline": roof, "clocks": clocks,
    }


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
