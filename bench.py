#!/usr/bin/env python
"""Benchmark: Taylor-exp scaling and squaring with mixed-precision Paterson--Stockmeyer.

Workload (one step): exp(A) for three seeded FP64 1024 x 1024 matrices with N(0,1) entries
rescaled to ||A||_1 = 0.5, 4 and 32 (0, 2 and 5 squarings), Taylor degree m = 30, s = 6,
evaluated by ``expm_taylor_ss`` through the C ABI.  The headline value is the mixed policy
(per-step precision by eq. (2.8), the last two Horner steps in the working precision) with
the working-precision products emulated on the tensor cores; the fixed-FP64 path
(Algorithm 2.1 on the FP64 pipe throughout) and the other policies are timed beside it,
and every policy's error is measured against the double-double oracle on sampled columns.

One JSON line on rank 0.  Under torchrun (N > 1) every rank evaluates its own copy of the
workload (independent replicas, no collective); value = evaluations of all ranks / slowest
rank's time.  ``--impl reference`` times the CPU oracle (plain double, all host cores) on
the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
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
C2_FORMATS = ("fp64", "bf16x3", "tf32", "bf16")
# dram__bytes_read.sum + dram__bytes_write.sum of one k_gemm_f64e<8> power-product launch at
# n = 1024 from the ncu capture summarised in profiles/gemm_f64e_n1024_bench.md (None until
# the current kernel has been captured)
F64E_N1024_DRAM_BYTES = 121.71e6
SEED = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpps", choices=["mpps", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--m", type=int, default=30)
    ap.add_argument("--policy", default="ns_e_mixp",
                    choices=["ns_e", "ns_e_mixp", "paper_e", "fixed_e", "ns", "paper", "fixed"],
                    help="headline policy (the others are timed beside it)")
    ap.add_argument("--policies", default="fixed,ns,fixed_e,ns_e,ns_e_mixp",
                    help="comma list of policies timed beside the headline (fixed is always kept)")
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error check")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the compact C3/C4/C5 results of the default line")
    ap.add_argument("--kernel", default=None,
                    choices=["gemm_f64", "gemm_bf16", "gemm_bf16x3", "gemm_tf32", "gemm_fp8",
                             "gemm_f64e9", "gemm_f64e8", "gemm_f64e6", "lu_solve_f64e8",
                             "lu_solve_f64"],
                    help="time one product kernel alone (mpps_matmul), or one linear solve "
                         "R = Q^-1 P (lu_solve: the Pade exp's solve), instead of the workload")
    ap.add_argument("--batch", type=int, default=1, help="batch for --kernel")
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c4", "c5"],
                    help="c2: exp n=1024 (the headline line); c3: 4096 uneven matrices; "
                         "c4: adjoint batch of 512 FP32 128x128; c5: Pade13 / cos at n=2048")
    return ap.parse_args()


def run_lu(args):
    """One linear solve R = Q^-1 P (Gaussian Q and P of order n) per step through lu_solve,
    timed with CUDA events around each call; 8 n^3 / 3 FP64 flops per solve (the LU and the
    two triangular solves with n right-hand sides)."""
    import numpy as np
    import torch

    import paper_2312_17396_gb300 as mpps
    from paper_2312_17396_gb300 import inputs
    dev = torch.device("cuda", 0)
    n = args.n
    pol = mpps.FIXED if args.kernel.endswith("_f64") else mpps.FIXED_E
    Q = torch.from_numpy(inputs.gaussian_batch(1, n, seed=1)).to(dev)
    P = torch.from_numpy(inputs.gaussian_batch(1, n, seed=2)).to(dev)
    R = torch.empty_like(P)
    for _ in range(args.warmup):
        mpps.lu_solve(Q, P, policy=pol, out=R)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mpps.lu_solve(Q, P, policy=pol, out=R)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    avg = float(np.mean(ms))
    print(json.dumps({"kernel": args.kernel, "n": n, "ms_per_solve": avg,
                      "fp64_equiv_tflops": 8.0 * n ** 3 / 3.0 / (avg / 1e3) / 1e12}), flush=True)


def run_kernel(args):
    """Single-product timing through mpps_matmul: CUDA events around each launch."""
    if args.kernel.startswith("lu_solve"):
        return run_lu(args)
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
    cls = (mpps.PROF_GEMM_F64 if fmt == "fp64" else
           mpps.PROF_GEMM_F64E if fmt.startswith("f64e") else mpps.PROF_GEMM_TC)
    mpps.profile_enable(True)
    mpps.profile_reset()
    for _ in range(args.steps):
        flush.fill_(1.0)
        mpps.matmul(A, B, fmt, out=C)
    torch.cuda.synchronize()
    launches, ms, _ = mpps.profile_read(cls)
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


POLICY_DESC = {
    "ns_e": "mixed (eq. (2.8), FP64 floors on steps 1-2), working-precision products emulated "
            "with 8 exact bf16 slices on tcgen05",
    "paper_e": "mixed (eq. (2.8) as in Algorithm 3.1), emulated working precision",
    "fixed_e": "fixed working precision, every product emulated (8 slices)",
    "ns": "mixed (eq. (2.8), FP64 floors on steps 1-2), working precision on the FP64 pipe",
    "paper": "mixed (eq. (2.8) as in Algorithm 3.1), FP64 pipe",
    "fixed": "fixed FP64 on the FP64 pipe (Algorithm 2.1 + eq. (3.6))",
    "ns_e_mixp": "ns_e with mixed-precision powers: power tree X^2, X^3, Y = X^3 X^3, leaves "
                 "X^4 = X^3 X and X^5 = X^3 X^2 in the slices the leaf rule allows",
}


def run_config(args, which=None, steps=None, warmup=None, emit=True):
    """The other workloads (mixed policy vs fixed FP64, errors against the oracle on a
    sample, the dominant kernel class's executed-flop roofline from a profiled pass): C3
    uneven batch, C4 adjoint batch, C5 n = 2048 general polynomials.  Prints one JSON line
    (emit) and returns it."""
    import numpy as np
    import torch

    import oracle
    import paper_2312_17396_gb300 as mpps
    from paper_2312_17396_gb300 import inputs

    which = which or args.config
    steps = steps or args.steps
    warmup = warmup if warmup is not None else args.warmup
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    mpps.lib()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    classes = (mpps.PROF_GEMM_F64, mpps.PROF_GEMM_F64E, mpps.PROF_GEMM_TC, mpps.PROF_SLICE,
               mpps.PROF_ELEMENTWISE)
    cname = {mpps.PROF_GEMM_F64: "k_gemm_f64 (DMMA)", mpps.PROF_GEMM_F64E: "k_gemm_f64e (tcgen05)",
             mpps.PROF_GEMM_TC: "k_gemm_tc (tcgen05)", mpps.PROF_SLICE: "slicing",
             mpps.PROF_ELEMENTWISE: "elementwise"}

    def roofline_of(step, step_ms, passes=2):
        """Per-class CUDA-event times of the library's launches over `passes` steps (a
        separate, profiled pass): the dominant class, its executed TFLOP/s and fraction."""
        mpps.profile_enable(True)
        mpps.profile_reset()
        for _ in range(passes):
            step()
        torch.cuda.synchronize()
        prof = {c: mpps.profile_read(c) for c in classes}
        mpps.profile_enable(False)
        mpps.profile_reset()
        products = (mpps.PROF_GEMM_F64, mpps.PROF_GEMM_F64E, mpps.PROF_GEMM_TC)
        dom = max(products, key=lambda c: prof[c][1])   # the dominant product class
        launches, ms, work = prof[dom]
        ach = work / (ms / 1e3) / 1e12 if ms > 0 and work > 0 else None
        peak, src = (peak_fp64_tflops() if dom == mpps.PROF_GEMM_F64 else peak_bf16_tflops(step_ms))
        # per-class event time per step (the classes overlap when launches run on several
        # streams, so the sum may exceed the step)
        return {"bound": "tensor", "kernel": cname[dom], "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": (ach / peak) if ach else None, "peak_source": src,
                "launches_per_step": launches // passes,
                "class_ms_per_step": {cname[c]: prof[c][1] / passes for c in classes}}

    def timed(step, steps, warmup):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    line = {"metric": METRIC, "unit": "evals/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "higher_is_better": True, "data": "synthetic",
            "impl": "mpps", "vs_baseline": None}
    if which == "c3":
        count = 4096
        mats, degs = inputs.uneven_batch(count, 8, 256, 0.1, 10.0, seed=3)
        dA = [torch.from_numpy(A).to(dev) for A in mats]
        res = {}
        # ||A||_1 <= 10: sigma <= 4, so five blind squaring steps cover every matrix and the
        # whole grouped call can be captured in a CUDA graph (nothing is read back)
        graph_pol = dataclasses.replace(mpps.NS_E, max_squarings=5)
        refs = {k: oracle.expm_ss_dd(mats[k], int(degs[k]), oracle.sigma_for(mats[k]))
                for k in range(0, count, count // 12)}   # the oracle on a sample, once
        for name, pol in (("ns_e", mpps.NS_E), ("ns_e_graph", graph_pol), ("fixed", mpps.FIXED)):
            outs = [torch.empty_like(a) for a in dA]
            _, reps = mpps.expm_grouped(dA, degs, policy=pol, outs=outs, report=True)
            if name == "ns_e_graph":
                g = torch.cuda.CUDAGraph()
                side = torch.cuda.Stream()
                side.wait_stream(stream)
                with torch.cuda.stream(side):
                    mpps.expm_grouped(dA, degs, policy=pol, outs=outs)
                stream.wait_stream(side)
                torch.cuda.synchronize()
                with torch.cuda.graph(g, capture_error_mode="relaxed"):
                    mpps.expm_grouped(dA, degs, policy=pol, outs=outs)
                fn = g.replay
            else:
                fn = (lambda pol=pol, outs=outs: mpps.expm_grouped(dA, degs, policy=pol, outs=outs))
            with ClockSampler(dev.index) as clk:
                ms = timed(fn, steps, max(3, warmup))
            flops = sum(2.0 * A.shape[0] ** 3 * sum(r["gemms"].values()) for A, r in zip(mats, reps))
            errs = [oracle.rel_err_1norm(outs[k].cpu().numpy(), eh, el) for k, (eh, el) in refs.items()]
            res[name] = {"evals_per_s": count / (ms / 1e3), "ms_per_step": ms,
                         "tflops": flops / (ms / 1e3) / 1e12, "max_rel_err_1norm_sampled": max(errs),
                         "clocks": clk.summary()}
        line["roofline"] = roofline_of(lambda: mpps.expm_grouped(dA, degs, policy=mpps.NS_E),
                                       res["ns_e"]["ms_per_step"])
        line.update({"value": res["ns_e"]["evals_per_s"], "ms_per_step": res["ns_e"]["ms_per_step"],
                     "dtype": "f64", "scaling": "weak",
                     "config": {"workload": "C3: 4096 matrices, n ~ U[8,256], ||A||_1 log-uniform in "
                                            "[0.1,10], Taylor-exp m in {12,18,24}, sigma per matrix; "
                                            "bucketed zero-padded batches planned on the GPU, buckets "
                                            "on forked streams", "policy": "ns_e",
                                "graph": "ns_e_graph: the same call captured once in a CUDA graph "
                                         "(max_squarings 5) and replayed"},
                     "policies": res})
    elif which == "c4":
        n, m, batch = 128, 18, 512
        rng = np.random.default_rng(4)
        A32 = torch.tensor(rng.standard_normal((batch, n, n)) / np.sqrt(n), dtype=torch.float32,
                           device=dev)
        G = torch.tensor(rng.standard_normal((batch, n, n)), dtype=torch.float32, device=dev)
        coef = mpps.taylor_exp_coeffs(m)
        res = {}
        step_of = {}
        grefs = {b: oracle.adjoint_dd(oracle.taylor_exp_rational(m), A32[b].double().cpu().numpy(),
                                      G[b].double().cpu().numpy()) for b in (0, batch // 2, batch - 1)}
        for name, pol in (("ns_e", mpps.NS_E), ("fixed", mpps.FIXED)):
            A = A32.clone().requires_grad_(True)

            def step(A=A, pol=pol):
                A.grad = None
                P = mpps.poly(A, coef, pol)
                P.backward(G)
            step_of[name] = step
            with ClockSampler(dev.index) as clk:
                ms = timed(step, steps, max(3, warmup))
            step()
            grad = A.grad.double().cpu().numpy()
            errs = [oracle.norm1(grad[b] - gh - gl) / oracle.norm1(gh) for b, (gh, gl) in grefs.items()]
            res[name] = {"evals_per_s": batch / (ms / 1e3), "ms_per_step": ms,
                         "max_rel_err_1norm_sampled": max(errs), "clocks": clk.summary()}
        line["roofline"] = roofline_of(step_of["ns_e"], res["ns_e"]["ms_per_step"])
        line.update({"value": res["ns_e"]["evals_per_s"], "ms_per_step": res["ns_e"]["ms_per_step"],
                     "unit": "gradients/s", "dtype": "f32 storage, f64 evaluation", "scaling": "weak",
                     "config": {"workload": "C4: 512 x 128x128 FP32, N(0,1)/sqrt(n), Taylor exp m=18 "
                                            "forward + adjoint through autograd", "policy": "ns_e"},
                     "policies": res})
    else:
        n = 2048
        A = inputs.prescribed_eigen_matrix(n, seed=5)
        B = A @ A                                    # the cosine's argument, formed on the host
        As = A / np.abs(A).sum(axis=0).max()         # labelled scaled variant, ||X||_1 = 1
        q, mc = 13, 16
        jobs = [("pade13_num", mpps.pade_exp_num_coeffs(q), oracle.pade_exp_num_rational(q), A),
                ("pade13_den", mpps.pade_exp_den_coeffs(q), oracle.pade_exp_den_rational(q), A),
                ("cos16_in_B", mpps.cos_taylor_coeffs(mc), oracle.cos_taylor_rational(mc), B),
                ("pade13_num_scaled", mpps.pade_exp_num_coeffs(q), oracle.pade_exp_num_rational(q), As)]
        cols = np.random.default_rng(7).choice(n, size=8, replace=False)
        V = np.zeros((n, cols.size)); V[cols, np.arange(cols.size)] = 1.0
        res = {}
        # all formats (FP8 tail blocks allowed); the working precision is F64E(9), 8 slices
        # with the pairs of order 8: at n = 2048 the 36-pair F64E(8) is about 2x less
        # accurate than an FP64 product on these inputs, F64E(9) below it
        pol_mixed = dataclasses.replace(mpps.NS_E, f64_slices=9)
        pol_fixed_e = dataclasses.replace(mpps.FIXED_E, f64_slices=9)
        for name, coef, rat, X in jobs:
            dX = torch.from_numpy(X).to(dev)
            rh, rl = oracle.ps_apply_dd(rat, X, V)
            ref = rh + rl
            entry = {}
            for pname, pol in (("ns_e", pol_mixed), ("fixed_e", pol_fixed_e), ("fixed", mpps.FIXED)):
                out = torch.empty_like(dX)
                _, rep = mpps.ps_eval(coef, dX, policy=pol, out=out, report=True)
                with ClockSampler(dev.index) as clk:
                    ms = timed(lambda: mpps.ps_eval(coef, dX, policy=pol, out=out), steps,
                               max(3, warmup))
                P = out.cpu().numpy()[:, cols]
                entry[pname] = {"evals_per_s": 1e3 / ms, "ms_per_step": ms,
                                "rel_err_1norm_sampled_cols": oracle.norm1(P - ref) / oracle.norm1(ref),
                                "formats": rep[0]["fmt"], "clocks": clk.summary()}
            res[name] = entry
        # the full [13/13] Pade exp (one power chain, LU solve, squarings), checked against
        # the emulated Taylor scaling and squaring of the same matrix
        dA = torch.from_numpy(A).to(dev)
        E_t = mpps.expm(dA, m=30, policy=pol_fixed_e)
        entry = {}
        for pname, pol in (("ns_e", pol_mixed), ("fixed", mpps.FIXED)):
            out = torch.empty_like(dA)
            mpps.expm_pade(dA, policy=pol, out=out)
            with ClockSampler(dev.index) as clk:
                ms = timed(lambda: mpps.expm_pade(dA, policy=pol, out=out), steps, max(3, warmup))
            d = ((out - E_t).abs().sum(dim=0).max() / E_t.abs().sum(dim=0).max()).item()
            entry[pname] = {"evals_per_s": 1e3 / ms, "ms_per_step": ms,
                            "rel_diff_1norm_vs_taylor_expm": d, "clocks": clk.summary()}
        res["expm_pade13"] = entry
        coef0, X0 = jobs[0][1], torch.from_numpy(jobs[0][3]).to(dev)
        line["roofline"] = roofline_of(lambda: mpps.ps_eval(coef0, X0, policy=pol_mixed),
                                       res["pade13_num"]["ns_e"]["ms_per_step"])
        tot_mixed = sum(res[j[0]]["ns_e"]["ms_per_step"] for j in jobs[:3])
        tot_fixed = sum(res[j[0]]["fixed"]["ms_per_step"] for j in jobs[:3])
        line.update({"value": 1e3 / tot_mixed, "ms_per_step": tot_mixed,
                     "unit": "evals/s (Pade13 num + den + cos16(B), one 2048 matrix)",
                     "dtype": "f64", "scaling": "weak", "fixed_value": 1e3 / tot_fixed,
                     "config": {"workload": "C5: n=2048 Q diag(lambda) Q^T, lambda ~ U[-8,8]; Pade[13/13] "
                                            "numerator and denominator (s=4) and Taylor cos of degree 16 "
                                            "in B = A^2; plus a scaled variant with ||X||_1 = 1",
                                "policy": "ns_e (all formats, f64_slices=9)"},
                     "jobs": res})
    if emit:
        print(json.dumps(line), flush=True)
    return line


def compact(line):
    """The headline fields of a config line: value, mixed over fixed, sampled errors,
    roofline."""
    out = {"workload": line["config"]["workload"], "value": line["value"], "unit": line["unit"],
           "ms_per_step": line["ms_per_step"], "roofline": line.get("roofline")}
    pol = line.get("policies")
    if pol:
        out["fixed_value"] = pol["fixed"]["evals_per_s"]
        out["mixed_over_fixed"] = line["value"] / pol["fixed"]["evals_per_s"]
        out["max_rel_err_mixed"] = pol["ns_e"]["max_rel_err_1norm_sampled"]
        out["max_rel_err_fixed"] = pol["fixed"]["max_rel_err_1norm_sampled"]
        if "ns_e_graph" in pol:
            out["graph_replay_value"] = pol["ns_e_graph"]["evals_per_s"]
    jobs = line.get("jobs")
    if jobs:
        out["fixed_value"] = line["fixed_value"]
        out["mixed_over_fixed"] = line["value"] / line["fixed_value"]
        out["rel_err_mixed"] = {k: v["ns_e"].get("rel_err_1norm_sampled_cols")
                                for k, v in jobs.items() if "rel_err_1norm_sampled_cols" in v["ns_e"]}
        out["rel_err_fixed"] = {k: v["fixed"].get("rel_err_1norm_sampled_cols")
                                for k, v in jobs.items() if "rel_err_1norm_sampled_cols" in v["fixed"]}
        if "expm_pade13" in jobs:
            out["expm_pade13"] = {k: {"evals_per_s": v["evals_per_s"],
                                      "rel_diff_vs_taylor": v["rel_diff_1norm_vs_taylor_expm"]}
                                  for k, v in jobs["expm_pade13"].items()}
    return out


def peak_bf16_tflops(step_ms):
    """Measured dense bf16 peak: the burst figure for a kernel inside a step of a few ms (the
    clocks stay at their maximum), the sustained one for steps of a second or more."""
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if step_ms < 100.0:
            return pk.get("bf16_tflops", 1900.0), "measured bf16 burst"
        return pk.get("bf16_tflops_sustained", 1700.0), "measured bf16 sustained"
    except Exception:
        return (1900.0, "fallback bf16 burst") if step_ms < 100.0 else (1700.0, "fallback bf16 sustained")


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
    if args.config != "c2":
        run_config(args)
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
    # the n = 1024 exp workload's mixed ladder is FP64 / 3xBF16 / TF32 / BF16 (no FP8 steps)
    c2 = dict(formats=C2_FORMATS)
    pols = {"ns_e": dataclasses.replace(mpps.NS_E, **c2),
            "ns_e_mixp": dataclasses.replace(mpps.NS_E, mixed_powers=True, **c2),
            "paper_e": dataclasses.replace(mpps.PAPER_E, **c2), "fixed_e": mpps.FIXED_E,
            "ns": dataclasses.replace(mpps.NS, **c2), "paper": dataclasses.replace(mpps.PAPER, **c2),
            "fixed": mpps.FIXED}
    head = args.policy
    extra = [p for p in args.policies.split(",") if p in pols]
    order = [head] + [p for p in dict.fromkeys(["fixed"] + extra) if p != head]
    mats = make_inputs(n)
    dA = [torch.from_numpy(A).to(dev) for A in mats]
    dS = torch.from_numpy(np.stack(mats)).to(dev)          # the step's batch: (3, n, n)
    outs = {p: torch.empty_like(dS) for p in order}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream(dev)
    classes = (mpps.PROF_GEMM_F64, mpps.PROF_GEMM_F64E, mpps.PROF_GEMM_TC, mpps.PROF_SLICE,
               mpps.PROF_ELEMENTWISE)
    cname = {mpps.PROF_GEMM_F64: "gemm_f64", mpps.PROF_GEMM_F64E: "gemm_f64e",
             mpps.PROF_GEMM_TC: "gemm_tc", mpps.PROF_SLICE: "slice",
             mpps.PROF_ELEMENTWISE: "elementwise"}

    def step(p, reports=None):
        """One pass over the batch: one expm call on the three matrices (each matrix keeps its
        own sigma and operand scales; a Horner step runs in the most precise format any of
        them asks for)."""
        if reports is not None:
            _, rep = mpps.expm(dS, m=m, policy=pols[p], out=outs[p], report=True)
            reports.extend(rep)
        else:
            mpps.expm(dS, m=m, policy=pols[p], out=outs[p])

    def timed(p, steps, profile):
        """Step times (CUDA events on the stream); with profile=True the library also records
        events around each of its launches (per-class kernel times), which adds work to the
        stream, so the headline time comes from an unprofiled pass."""
        times = []
        if profile:
            mpps.profile_enable(True)
            mpps.profile_reset()
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(p)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = None
        if profile:
            prof = {c: mpps.profile_read(c) for c in classes}
            mpps.profile_enable(False)
            mpps.profile_reset()
        return times, prof

    reps = {}
    for p in order:
        reps[p] = []
        step(p, reps[p])
        for _ in range(max(0, args.warmup - 1)):
            step(p)
    torch.cuda.synchronize()

    results = {}
    clk = None
    for p in order:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if p == head:
            with ClockSampler(dev.index) as clk:
                t, _ = timed(p, args.steps, False)
        else:
            t, _ = timed(p, args.steps, False)
        _, prof = timed(p, args.steps, True)          # per-class kernel times, separate pass
        torch.cuda.synchronize()
        ms = sum(t) / len(t)
        if dist:
            tt = torch.tensor([ms], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms = float(tt[0])
        prods = sum(sum(v for k, v in R["gemms"].items()) for R in reps[p])
        results[p] = {"evals_per_s": len(dA) * world / (ms / 1e3), "ms_per_step": ms,
                      "tflops_fp64_equiv": prods * 2.0 * n ** 3 * world / (ms / 1e3) / 1e12,
                      "kernels": {cname[c]: {"launches": prof[c][0] // args.steps,
                                             "ms_per_step": prof[c][1] / args.steps,
                                             "executed_tflops": (prof[c][2] / prof[c][1] / 1e9)
                                             if prof[c][1] > 0 and prof[c][2] > 0 else None}
                                  for c in classes},
                      "formats": [R["fmt"][1:] for R in reps[p]],
                      "pow_fmt": [R["pow_fmt"][2:] for R in reps[p]],
                      "policy": POLICY_DESC[p], "_prof": prof}

    # the same three evaluations as three separate calls, one matrix each (each matrix then
    # runs its own plan, and each product has 128 tiles for 152 SMs): reported beside the
    # batched headline
    sep = None
    if world == 1:
        souts = [torch.empty_like(a) for a in dA]

        def step_separate():
            for k in range(len(dA)):
                mpps.expm(dA[k], m=m, policy=pols[head], out=souts[k])

        for _ in range(max(3, args.warmup)):
            step_separate()
        torch.cuda.synchronize()
        ct = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step_separate()
            e1.record(stream)
            e1.synchronize()
            ct.append(e0.elapsed_time(e1))
        sms = sum(ct) / len(ct)
        sep = {"value": len(dA) / (sms / 1e3), "unit": "evals/s", "ms_per_step": sms,
               "policy": head + ", one call per matrix",
               "max_rel_diff_vs_batched": max(float((souts[k] - outs[head][k]).abs().max() /
                                                    outs[head][k].abs().max())
                                              for k in range(len(dA)))}

    # e2e: a pinned host batch through the C ABI (H2D + D2H inside the timed region), headline
    # policy, one call per step; the torch tensor owns the page-locked memory the numpy views
    # point at
    pinned = [torch.empty((len(mats), n, n), dtype=torch.float64, pin_memory=True) for _ in (0, 1)]
    host_in, host_out = pinned[0].numpy(), pinned[1].numpy()
    host_in[...] = np.stack(mats)
    mpps.expm(host_in, m=m, policy=pols[head], out=host_out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mpps.expm(host_in, m=m, policy=pols[head], out=host_out)
    e2e_s = time.perf_counter() - t0
    e2e_value = len(mats) * args.steps * world / e2e_s

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    errs = None
    if not args.no_check:
        import oracle
        cols = [0, n // 2, n - 1]
        torch.cuda.synchronize()
        errs = {p: [] for p in order}
        for k, A in enumerate(mats):
            sg = oracle.sigma_for(A)
            V = np.zeros((n, len(cols)))
            for t, j in enumerate(cols):
                V[j, t] = 1.0
            wh, wl = oracle.ps_apply_dd(oracle.taylor_exp_rational(m), np.ldexp(A, -sg), V, 2 ** sg)
            ref = np.abs(wh).sum(axis=0)
            for p in order:
                E = outs[p][k].cpu().numpy()
                errs[p].append(float(np.max(np.abs(E[:, cols] - wh - wl).sum(axis=0) / ref)))
        for p in order:
            results[p]["rel_err_1norm_sampled"] = errs[p]

    # the acceptance rule: every mixed policy's sampled error <= 2 x the fixed-FP64 error of the
    # same column, up to a floor of 4 ulps of ||P||
    within2x = None
    if errs is not None:
        within2x = all(e <= 2.0 * f + 4 * 2.0 ** -53 for p in order if p not in ("fixed", "fixed_e")
                       for e, f in zip(errs[p], errs["fixed"]))

    # roofline of the headline path's dominant kernel class
    hp = results[head]["_prof"]
    dom = max(classes, key=lambda c: hp[c][1])
    launches, ms_tot, work = hp[dom]
    achieved = work / (ms_tot / 1e3) / 1e12 if ms_tot > 0 else 0.0
    if dom == mpps.PROF_GEMM_F64:
        peak, src = peak_fp64_tflops()
        kern = "k_gemm_f64 (DMMA m16n8k4 f64)"
    else:
        peak, src = peak_bf16_tflops(results[head]["ms_per_step"])
        kern = ("k_gemm_f64e (tcgen05 kind::f16, exact bf16 slice products; achieved counts "
                "executed bf16 flops)" if dom == mpps.PROF_GEMM_F64E else "k_gemm_tc (tcgen05)")
    step_ms_tot = results[head]["ms_per_step"] * args.steps
    # DRAM bytes (read + write) of one launch of the dominant kernel, from the ncu capture
    # summarised in profiles/ (null when no capture of the current kernel at this size exists)
    traffic, traffic_src = None, None
    if dom == mpps.PROF_GEMM_F64E and n == 1024 and F64E_N1024_DRAM_BYTES is not None:
        traffic = F64E_N1024_DRAM_BYTES
        traffic_src = "profiles/gemm_f64e_n1024_bench.md (one power-product launch of the batch)"
    roofline = {"bound": "tensor", "kernel": kern, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch", "traffic_source": traffic_src,
                "peak_source": src,
                "share_of_step": ms_tot / step_ms_tot, "launches_per_step": launches // args.steps}
    for p in order:
        results[p].pop("_prof")

    value = results[head]["evals_per_s"]
    fixed_value = results["fixed"]["evals_per_s"]
    gpu_launches = sum(results[head]["kernels"][k]["launches"] for k in results[head]["kernels"]) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": results[head]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (mixed: bf16 tensor-core slices and low-precision Horner products)",
        "data": "synthetic",
        "config": {"workload": f"expm_taylor_ss n={n} m={m} s=6, a batch of three matrices at "
                               f"||A||_1 in {list(NORMS)} (sigma 0/2/5), N(0,1) entries, seed {SEED}+k; "
                               "one batched call per step",
                   "policy": head, "formats": "+".join(C2_FORMATS),
                   "l2": "flushed (256 MiB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "tflops": results[head]["tflops_fp64_equiv"],
        "fixed": {"value": fixed_value, "unit": "evals/s", "ms_per_step": results["fixed"]["ms_per_step"],
                  "tflops": results["fixed"]["tflops_fp64_equiv"], "policy": POLICY_DESC["fixed"]},
        "speedup_vs_fixed": value / fixed_value,
        # the precision rule's own gain, like for like: mixed over fixed on the same engine
        "mixed_over_fixed_same_engine": {
            "emulated (ns_e / fixed_e)": (results["ns_e"]["evals_per_s"] /
                                          results["fixed_e"]["evals_per_s"])
            if "ns_e" in results and "fixed_e" in results else None,
            "emulated with mixed powers (ns_e_mixp / fixed_e)":
                (results["ns_e_mixp"]["evals_per_s"] / results["fixed_e"]["evals_per_s"])
            if "ns_e_mixp" in results and "fixed_e" in results else None,
            "fp64_pipe (ns / fixed)": (results["ns"]["evals_per_s"] / fixed_value)
            if "ns" in results else None},
        "mixed_within_2x_fixed_error": within2x,
        # the mixed precision inside the powers (power tree, leaves in fewer slices): its
        # measured gain over the same policy with every power in the working precision
        "mixed_powers": ({"value": results["ns_e_mixp"]["evals_per_s"],
                          "gain_over_ns_e": results["ns_e_mixp"]["evals_per_s"] /
                          results["ns_e"]["evals_per_s"],
                          "leaf_formats": results["ns_e_mixp"].get("pow_fmt"),
                          "rel_err_1norm_sampled": results["ns_e_mixp"].get("rel_err_1norm_sampled")}
                         if "ns_e_mixp" in results and "ns_e" in results else None),
        "policies": results,
        "per_matrix_calls": sep,
        "roofline": roofline,
        "gpu_launches": int(gpu_launches),
        "e2e": {"value": e2e_value, "unit": "evals/s",
                "h2d_bytes_per_step": len(mats) * n * n * 8,
                "d2h_bytes_per_step": len(mats) * n * n * 8, "host_buffers": "pinned"},
        "clocks": clk.summary() if clk else None,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(n, m, mats)
    if not args.no_configs and world == 1:
        # the other workloads, compact, in the same line (fewer steps: a bounded run time)
        line["configs"] = {}
        for c in ("c3", "c4", "c5"):
            try:
                line["configs"][c] = compact(run_config(args, c, steps=3, warmup=2, emit=False))
            except Exception as exc:   # pragma: no cover - reported, not hidden
                line["configs"][c] = {"error": repr(exc)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
