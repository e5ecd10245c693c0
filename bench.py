#!/usr/bin/env python
"""Benchmark: Taylor-exp scaling and squaring with mixed-precision Paterson--Stockmeyer.

Workload (one step): exp(A) for three seeded FP64 1024 x 1024 matrices with N(0,1) entries
rescaled to ||A||_1 = 0.5, 4 and 32 (0, 2 and 5 squarings), Taylor degree m = 30, s = 6,
evaluated by ``expm_taylor_ss`` through the C ABI.  The headline value is the mixed
policy (per-step precision by eq. (2.8), FP64 floors on the last two Horner steps); the
fixed-FP64 path (Algorithm 2.1 in FP64 throughout) is timed beside it, and both errors are
measured against the double-double oracle on sampled columns.

One JSON line on rank 0.  Under torchrun (N > 1) every rank evaluates its own copy of the
workload (independent replicas, no collective); value = evaluations of all ranks / slowest
rank's time.  ``--impl reference`` times the CPU oracle (plain double, all host cores) on
the same workload instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p(A) evals/s and TFLOP/s, mixed vs fixed FP64 PS, at equal 1-norm rel. error"
NORMS = (0.5, 4.0, 32.0)
SEED = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpps", choices=["mpps", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--m", type=int, default=30)
    ap.add_argument("--policy", default="ns", choices=["ns", "paper", "fixed"])
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error check")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default=None,
                    choices=["gemm_f64", "gemm_bf16", "gemm_bf16x3", "gemm_tf32", "gemm_fp8"],
                    help="time one product kernel alone (mpps_matmul) instead of the workload")
    ap.add_argument("--batch", type=int, default=1, help="batch for --kernel")
    return ap.parse_args()


def run_kernel(args):
    """Single-product timing through mpps_matmul: CUDA events around each launch."""
    import numpy as np
    import torch

    import paper_2312_17396_gb300 as mpps
    from paper_2312_17396_gb300 import inputs
    dev = torch.device("cuda", 0)
    fmt = {"f64": "fp64"}.get(args.kernel.split("_", 1)[1], args.kernel.split("_", 1)[1])
    n, b = args.n, args.batch
    A = torch.from_numpy(inputs.gaussian_batch(b, n, seed=1)).to(dev)
    B = torch.from_numpy(inputs.gaussian_batch(b, n, seed=2)).to(dev)
    C = torch.empty_like(A)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        mpps.matmul(A, B, fmt, out=C)
    torch.cuda.synchronize()
    cls = mpps.PROF_GEMM_F64 if fmt == "fp64" else mpps.PROF_GEMM_TC
    mpps.profile_enable(True)
    mpps.profile_reset()
    for _ in range(args.steps):
        flush.fill_(1.0)
        mpps.matmul(A, B, fmt, out=C)
    torch.cuda.synchronize()
    launches, ms = mpps.profile_read(cls)
    mpps.profile_enable(False)
    avg = ms / max(1, launches)
    tflops = 2.0 * n ** 3 * b / (avg / 1e3) / 1e12
    print(json.dumps({"kernel": args.kernel, "n": n, "batch": b, "launches": launches,
                      "ms_per_launch": avg, "tflops": tflops}), flush=True)


def peak_fp64_tflops():
    """FP64 tensor peak: the measured bf16 figure times the nominal FP64/BF16 ratio
    (1.25 / 2250 TFLOP/s), sustained figure for a kernel timed inside a long step."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        pk = json.load(open(path))
        return pk.get("bf16_tflops_sustained", 1700.0) * 1.25 / 2250.0, "measured bf16 sustained x 1.25/2250"
    except Exception:
        return 1700.0 * 1.25 / 2250.0, "fallback bf16 sustained x 1.25/2250"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(n):
    from paper_2312_17396_gb300 import inputs
    return [inputs.gaussian_matrix(n, seed=SEED + k, norm1=nrm) for k, nrm in enumerate(NORMS)]


def cpu_baseline(n, m, mats):
    """The oracle's plain-double scaling and squaring (Algorithm 2.1 + eq. (3.6)) on the host
    cores, on a bounded sample: one evaluation of the ||A||_1 = 4 matrix."""
    import oracle
    A = mats[1]
    sg = oracle.sigma_for(A)
    t0 = time.perf_counter()
    oracle.expm_ss_d(A, m, sg)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "evals/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"1 evaluation of exp(A), n={n}, m={m}, ||A||_1=4 (sigma={sg}), plain double "
                      f"({dt:.2f} s)"}


def run_reference(args, rank, world):
    import oracle
    n, m = args.n, args.m
    if rank != 0:
        return
    mats = make_inputs(n)
    oracle.build()
    times = []
    for it in range(args.warmup + args.steps):
        A = mats[it % 3]
        sg = oracle.sigma_for(A)
        t0 = time.perf_counter()
        oracle.expm_ss_d(A, m, sg)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = len(times) / tot
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"expm_taylor_ss n={n} m={m}, ||A||_1 in {list(NORMS)}",
                       "step": "one matrix per step, cycling through the three norms"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": "plain-double oracle, one exp(A) per step"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.kernel:
        run_kernel(args)
        return

    import numpy as np
    import torch

    import paper_2312_17396_gb300 as mpps

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    mpps.lib()
    n, m = args.n, args.m
    pol = {"ns": mpps.NS, "paper": mpps.PAPER, "fixed": mpps.FIXED}[args.policy]
    mats = make_inputs(n)
    dA = [torch.from_numpy(A).to(dev) for A in mats]
    dE = [torch.empty_like(a) for a in dA]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream(dev)

    def step(policy, reports=None):
        for k in range(len(dA)):
            if reports is not None:
                _, rep = mpps.expm(dA[k], m=m, policy=policy, out=dE[k], report=True)
                reports.append(rep[0])
            else:
                mpps.expm(dA[k], m=m, policy=policy, out=dE[k])

    def timed(policy, steps, sampler=None, profile=False):
        times = []
        if profile:
            mpps.profile_enable(True)
            mpps.profile_reset()
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(policy)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = None
        if profile:
            prof = {c: mpps.profile_read(c) for c in (mpps.PROF_GEMM_F64, mpps.PROF_GEMM_TC,
                                                      mpps.PROF_ELEMENTWISE)}
            mpps.profile_enable(False)
            mpps.profile_reset()
        return times, prof

    # warm-up (both policies), reports for the flop counts
    reps_mixed, reps_fixed = [], []
    step(pol, reps_mixed)
    step(mpps.FIXED, reps_fixed)
    for _ in range(max(0, args.warmup - 1)):
        step(pol); step(mpps.FIXED)
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t_mixed, prof = timed(pol, args.steps, profile=True)
    torch.cuda.synchronize()
    t_fixed, _ = timed(mpps.FIXED, args.steps)
    torch.cuda.synchronize()

    ms_mixed = sum(t_mixed) / len(t_mixed)
    ms_fixed = sum(t_fixed) / len(t_fixed)
    if dist:
        tt = torch.tensor([ms_mixed, ms_fixed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_mixed, ms_fixed = float(tt[0]), float(tt[1])
    evals = len(dA) * world
    value = evals / (ms_mixed / 1e3)
    fixed_value = evals / (ms_fixed / 1e3)

    def flops(reps):
        tot = 0
        for R in reps:
            g = sum(v for k, v in R["gemms"].items() if k != "squarings") + R["gemms"]["squarings"]
            tot += g * 2.0 * n ** 3
        return tot

    tflops_mixed = flops(reps_mixed) * world / (ms_mixed / 1e3) / 1e12
    tflops_fixed = flops(reps_fixed) * world / (ms_fixed / 1e3) / 1e12

    # e2e: host buffers through the C ABI (H2D + D2H inside the timed region)
    host_in = [np.ascontiguousarray(A) for A in mats]
    host_out = [np.empty_like(A) for A in mats]
    for k in range(len(mats)):
        mpps.expm(host_in[k], m=m, policy=pol, out=host_out[k])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for k in range(len(mats)):
            mpps.expm(host_in[k], m=m, policy=pol, out=host_out[k])
    e2e_s = time.perf_counter() - t0
    e2e_value = len(mats) * args.steps * world / e2e_s

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    # dominant kernel: the FP64 product (powers, early Horner steps, squarings)
    f64_launches, f64_ms = prof[mpps.PROF_GEMM_F64]
    tc_launches, tc_ms = prof[mpps.PROF_GEMM_TC]
    el_launches, el_ms = prof[mpps.PROF_ELEMENTWISE]
    peak, peak_src = peak_fp64_tflops()
    avg_f64 = f64_ms / max(1, f64_launches)
    achieved = 2.0 * n ** 3 / (avg_f64 / 1e3) / 1e12
    roofline = {"bound": "tensor", "kernel": "k_gemm_f64 (DMMA m16n8k4 f64)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": peak_src,
                "share_of_step": f64_ms / max(1e-9, sum(t_mixed))}

    errs = None
    if not args.no_check:
        import oracle
        cols = [0, n // 2, n - 1]
        errs = {"mixed": [], "fixed": []}
        E_mixed = [e.cpu().numpy() for e in dE]
        step(mpps.FIXED)
        torch.cuda.synchronize()
        E_fixed = [e.cpu().numpy() for e in dE]
        for k, A in enumerate(mats):
            sg = oracle.sigma_for(A)
            V = np.zeros((n, len(cols)))
            for t, j in enumerate(cols):
                V[j, t] = 1.0
            wh, wl = oracle.ps_apply_dd(oracle.taylor_exp_rational(m), np.ldexp(A, -sg), V, 2 ** sg)
            ref = np.abs(wh).sum(axis=0)
            for name, E in (("mixed", E_mixed[k]), ("fixed", E_fixed[k])):
                errs[name].append(float(np.max(np.abs(E[:, cols] - wh - wl).sum(axis=0) / ref)))

    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mixed,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (mixed: low-precision tensor-core Horner products)", "data": "synthetic",
        "config": {"workload": f"expm_taylor_ss n={n} m={m} s=6, one matrix each at "
                               f"||A||_1 in {list(NORMS)} (sigma 0/2/5), N(0,1) entries, seed {SEED}+k",
                   "policy": args.policy, "l2": "flushed (256 MiB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "tflops": tflops_mixed,
        "fixed": {"value": fixed_value, "unit": "evals/s", "ms_per_step": ms_fixed,
                  "tflops": tflops_fixed},
        "speedup_vs_fixed": value / fixed_value,
        "rel_err_1norm_sampled": errs,
        "formats": [R["fmt"][1:] for R in reps_mixed],
        "roofline": roofline,
        "kernels_ms_per_step": {"gemm_f64": f64_ms / args.steps, "gemm_tc": tc_ms / args.steps,
                                "elementwise": el_ms / args.steps},
        "gpu_launches": int(f64_launches + tc_launches + el_launches),
        "e2e": {"value": e2e_value, "unit": "evals/s",
                "h2d_bytes_per_step": len(mats) * n * n * 8,
                "d2h_bytes_per_step": len(mats) * n * n * 8},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(n, m, mats)
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
