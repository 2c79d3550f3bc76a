#!/usr/bin/env python3
"""Benchmark of the randUTV / powerURV hot path on GB300.

One step = one randUTV_basic (Algorithm 3) and one powerURV (Algorithm 1) factorization, FP64, of an
8192 x 8192 matrix A = Q1 diag(s) Q2^T with s_j = 10^(-8j/n) for j < n/2 and 1e-4 after, b = 128,
q = 1 (the 8192^2 configuration).  The metric is factorizations/s (two per step per GPU) with TFLOP/s
by the algorithmic flop model alongside.  A is 512 MB, larger than the 129 MB L2, so no flush is
needed between steps.  Multi-GPU runs are independent replicas (one matrix per rank, weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factorizations/s (randUTV + powerURV, FP64, 8192^2, b=128, q=1)"
WORKLOAD = "randUTV_basic + powerURV on 8192x8192 A = Q1 diag(s) Q2^T, s_j = 10^(-8j/n) (j < n/2) then 1e-4"
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel, taken from ncu captures
# summarised under profiles/ (figures copied from those files, not measured by this script).  Each entry
# names the source file of the kernel and the sha1 of its code (source_sha1: comments and blank lines
# removed) when the capture was taken; when the code has changed since, the figure no longer describes
# the kernel and the line reports traffic as null.
KERNEL_TRAFFIC = {
    "ozaki_gemm_4096": {"source": "gemm_ozaki.cu", "bytes_per_launch": 2692.4e6,
                        "kernel_sha1": "22b0be53d7c17448df989afd2bbd60402a74adf1",
                        "profile": "profiles/ozaki_gemm_kernel_4096.md"},
    "ozaki_step_8192": {"source": "gemm_ozaki.cu", "bytes_per_launch": 263.5e6,
                        "kernel_sha1": "22b0be53d7c17448df989afd2bbd60402a74adf1",
                        "profile": "profiles/kernel_dram_8192_step.md"},
    "panel_step_8192": {"source": "panel_qr.cu", "bytes_per_launch": 4.4e6,
                        "kernel_sha1": "562da21b6e4a15c7f25d40f97605d5b3c9c08b1f",
                        "profile": "profiles/kernel_dram_8192_step.md"},
}
# FP64 peak of the DFMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (measured 1.19 TFLOP/s at 1995 MHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--b", type=int, default=128)
    p.add_argument("--q", type=int, default=1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-accuracy", action="store_true")
    p.add_argument("--cpu-pow-n", type=int, default=2048, help="size of the matrix powerURV is timed on (oracle)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the learned-q + BF16-sketch and randUTV_boosted sub-results of the default line")
    p.add_argument("--plain-reps", type=int, default=3, help="runs of the plain FP64 comparison per method")
    p.add_argument("--methods", default="randutv,powerurv", help="comma list (profiling runs may time one)")
    p.add_argument("--gemm", default="auto", choices=["auto", "native", "emulated"],
                   help="FP64 products: library default, DFMA only, or emulated on the BF16 tensor cores")
    p.add_argument("--no-plain", action="store_true", help="skip the plain-FP64 (DFMA) comparison run")
    p.add_argument("--no-per-method", action="store_true", help="skip the per-method timing runs (profiling)")
    p.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "gemm", "boosted"],
                   help="c2: FP64 randUTV + powerURV 8192^2 (default); c3: BF16-sketch randUTV 16384^2, b=256, q=2; "
                        "c4: 512 uneven FP32 powerURV in one graph; c5: learned q + BF16 sketch, 8192^2, b=128; "
                        "gemm: the dominant kernel alone (FP64 GEMM 4096^3 emulated on the tensor cores); "
                        "boosted: randUTV_boosted 8192^2, b=128, q=--boost-q, p=--oversample")
    p.add_argument("--oversample", type=int, default=128, help="p of the boosted workload")
    p.add_argument("--boost-q", type=int, default=5, help="q of the boosted workload")
    return p.parse_args()


def source_sha1(name: str, text: str | None = None) -> str:
    """sha1 of a kernel source's code: comments, trailing blanks and empty lines removed, so that only a
    change of the code itself withdraws a recorded figure."""
    import hashlib
    import re
    if text is None:
        with open(os.path.join(ROOT, "paper_2106_13402_gb300", "csrc", name), encoding="utf-8") as f:
            text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha1("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def kernel_traffic(which: str):
    """(bytes per launch, source) of the recorded ncu capture, or (None, why) when there is none for the
    kernel as it is now."""
    t = KERNEL_TRAFFIC[which]
    if t["bytes_per_launch"] is None:
        return None, "no capture recorded"
    if t["kernel_sha1"] != source_sha1(t["source"]):
        return None, f"kernel changed since {t['profile']}"
    return t["bytes_per_launch"], f"ncu capture, {t['profile']} (copied, not measured here)"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------------------------ clock sampling --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return self.summarize(lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, max clock and the throttle reasons seen, from nvidia-smi CSV lines
        (FIELDS order, no header, no units); None without a usable sample."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------- helpers --
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (the slowest replica's time); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of independent replicas: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def step_flops(n, b, q):
    from paper_2106_13402_gb300 import testmats
    return testmats.flops_randutv(n, n, b, q) + testmats.flops_powerurv(n, n, q)


def cpu_rates(A_np, n, b, q, pow_n, pow_rate=None):
    """The oracle as it stands on the host cores, on a bounded sample of the step: randUTV's first step
    of the same n x n matrix (its public entry point with max_steps = 1), and, unless its rate is given,
    powerURV in full on a pow_n x pow_n matrix of the same recipe.  Returns the measured seconds and each
    method's rate (flop model / seconds)."""
    import oracle
    from paper_2106_13402_gb300 import testmats

    f_rand = testmats.flops_randutv(n, n, b, q, max_steps=1)
    t0 = time.perf_counter()
    oracle.randutv(A_np, b, q, seed=17, max_steps=1)
    t_rand = time.perf_counter() - t0
    out = {"randutv_s": t_rand, "randutv_rate": f_rand / t_rand, "randutv_gflop": f_rand / 1e9}
    if pow_rate is None:
        Ap, _ = testmats.make_matrix(pow_n, pow_n, "c2", 11, 12, device="cpu")
        f_pow = testmats.flops_powerurv(pow_n, pow_n, q)
        t0 = time.perf_counter()
        oracle.powerurv(Ap, q, seed=17)
        t_pow = time.perf_counter() - t0
        out.update(powerurv_s=t_pow, powerurv_rate=f_pow / t_pow, powerurv_gflop=f_pow / 1e9)
    else:
        out.update(powerurv_s=0.0, powerurv_rate=pow_rate, powerurv_gflop=0.0)
    return out


def cpu_extrapolate(r, n, b, q):
    """Seconds of one randUTV + powerURV step at n x n at the sampled rates (flop model)."""
    from paper_2106_13402_gb300 import testmats
    return testmats.flops_randutv(n, n, b, q) / r["randutv_rate"] + testmats.flops_powerurv(n, n, q) / r["powerurv_rate"]


def cpu_sample_text(r, n, b, q, pow_n):
    return (f"randUTV: its first step (of {n // b}) on the same {n}x{n} matrix, {r['randutv_gflop']:.0f} GFLOP in "
            f"{r['randutv_s']:.1f} s ({r['randutv_rate'] / 1e9:.2f} GFLOP/s); powerURV: in full on a {pow_n}x{pow_n} "
            f"matrix of the same recipe ({r['powerurv_rate'] / 1e9:.2f} GFLOP/s); each rate extrapolated to the "
            f"{n}x{n} method by the flop model")


def cpu_sample(A_np, n, b, q, pow_n):
    import oracle
    r = cpu_rates(A_np, n, b, q, pow_n)
    per_step_s = cpu_extrapolate(r, n, b, q)
    return {"value": 2.0 / per_step_s, "unit": "factorizations/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": cpu_sample_text(r, n, b, q, pow_n), "extrapolated": True,
            "seconds": round(r["randutv_s"] + r["powerurv_s"], 2)}


def power_norm(torch, M, iters=60):
    """Spectral norm estimate of M (power iteration on M^T M), FP64 on the GPU."""
    g = torch.Generator(device=M.device)
    g.manual_seed(5)
    x = torch.randn(M.shape[1], 1, generator=g, device=M.device, dtype=M.dtype)
    x /= torch.linalg.norm(x)
    s = torch.zeros((), device=M.device, dtype=M.dtype)
    for _ in range(iters):
        y = M.t() @ (M @ x)
        s = torch.linalg.norm(y)
        x = y / s
    return float(torch.sqrt(s))


# ------------------------------------------------------------------------------------------ our arm --
def _event_ms(torch, fn, stream):
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    fn()
    a1.record(stream)
    a1.synchronize()
    return a0.elapsed_time(a1)


def dominant_kernel_roofline(rrf, ms_step, steps, peaks, peak_src):
    """Read the event profiler (after rrf_gemm_profile_end) and describe the kernels it timed; the one with the
    largest share of the step is `roofline`, the others ride along under `others`."""
    gemm_ms, gemm_flops, gemm_launches = rrf.gemm_profile_end()
    emu_ms, emu_flops, emu_tflops, emu_launches = rrf.gemm_profile_emulated()
    emu_bytes = rrf.gemm_profile_emulated_bytes()
    pan_ms, pan_flops, pan_bytes, pan_launches = rrf.gemm_profile_panel()
    fp64_src = "152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe; recipe nominal 1.25)"
    kernels = []
    if emu_ms > 0:
        # the emulated GEMM's tensor-core kernel (BF16 digit products, timed inside a long step -> the
        # sustained BF16 peak)
        achieved = emu_tflops / (emu_ms / 1e3) / 1e12
        peak = float(peaks["bf16_tflops_sustained"])
        traffic, tsrc = kernel_traffic("ozaki_step_8192")
        kernels.append((emu_ms, {
            "kernel": "ozaki_gemm_kernel (FP64 product emulated with 7 BF16 digit slices)", "bound": "tensor",
            "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "traffic": traffic, "traffic_source": tsrc,
            "traffic_unit": "DRAM bytes read + written per launch, averaged over the launches of one step",
            "algorithmic_bytes_per_launch": round(emu_bytes / max(emu_launches, 1)),
            "achieved_gbs_algorithmic": round(emu_bytes / (emu_ms / 1e3) / 1e9, 1),
            "peak_source": f"{peak_src} bf16_tflops_sustained (MEASURED_PEAKS.json)",
            "work": "28 digit-pair products x 2 M N K' BF16 flops per launch (K' = K rounded up to 32)",
            "fp64_equivalent_tflops": round(emu_flops / (emu_ms / 1e3) / 1e12, 3),
            "launches": int(emu_launches), "avg_launch_ms": round(emu_ms / max(emu_launches, 1), 4),
            "share_of_step": round(emu_ms / (ms_step * steps), 4)}))
    if pan_ms > 0:
        achieved = pan_flops / (pan_ms / 1e3) / 1e12
        ptraffic, ptsrc = kernel_traffic("panel_step_8192")
        kernels.append((pan_ms, {
            "kernel": "panel_qr_kernel (Householder panel, one grid-wide reduction per column)", "bound": "alu",
            "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
            "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": ptraffic, "traffic_source": ptsrc,
            "traffic_unit": "DRAM bytes read + written per launch, averaged over the launches of one step",
            "work": "HQR flops 2 r w^2 - 2 w^3 / 3 per launch on the FP64 pipe (latency-bound: one grid barrier per column)",
            "algorithmic_bytes_per_launch": round(pan_bytes / max(pan_launches, 1)),
            "achieved_gbs_algorithmic": round(pan_bytes / (pan_ms / 1e3) / 1e9, 1),
            "peak_source": fp64_src, "launches": int(pan_launches),
            "avg_launch_ms": round(pan_ms / max(pan_launches, 1), 4), "share_of_step": round(pan_ms / (ms_step * steps), 4)}))
    if gemm_ms > 0:
        achieved = gemm_flops / (gemm_ms / 1e3) / 1e12
        kernels.append((gemm_ms, {
            "kernel": "gemm_f64_kernel (+ split-K reduction)", "bound": "alu", "achieved": round(achieved, 4),
            "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
            "traffic": None, "peak_source": fp64_src, "launches": int(gemm_launches),
            "avg_launch_ms": round(gemm_ms / max(gemm_launches, 1), 4),
            "share_of_step": round(gemm_ms / (ms_step * steps), 4)}))
    if not kernels:
        return {"kernel": None, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "note": "no profiled launch in the pass", "others": []}
    kernels.sort(key=lambda t: -t[0])
    roof = dict(kernels[0][1])
    roof["others"] = [k for _, k in kernels[1:]]
    return roof


def extras_8192(torch, rrf, testmats, A, s, dev, n, b):
    """Sub-results for the configurations the speed-up target is set on, on the same 8192^2 matrix:
    (1) learned per-step q with the BF16 sketch (fallback q = 2) against the plain FP64 method with q = 2;
    (2) randUTV_basic with q = 10 and (3) randUTV_boosted (Algorithm 2, q = 5, p = b), each against the same
    algorithm with every product on the DFMA pipe: both meet e_k <= 1.1 sigma_{k+1} at every boundary.  One warm run and one timed run each; e_k / sigma_{k+1} at every block boundary."""
    from paper_2106_13402_gb300 import qpolicy
    ks = list(range(b, n, b))
    steps = n // b
    out = (rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev))
    stream = torch.cuda.current_stream()
    on_target = lambda r: sum(1 for v in r.values() if v <= 1.1)

    def timed(opts, q=2):
        ws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, opts), dev)
        rrf.randutv(A, b, q, 17, opts=opts, ws=ws, out=out)
        t = _event_ms(torch, lambda: rrf.randutv(A, b, q, 17, opts=opts, ws=ws, out=out, check_status=False), stream)
        st = rrf.lib().rrf_workspace_status(rrf._vp(ws.data_ptr()), rrf._stream(None))
        r = _boundary_ratios(torch, out[1], s, b, ks)
        del ws
        return t, r, int(st)

    res = {}
    pms, r_plain, _ = timed(rrf.make_opts(gemm_mode=rrf.GEMM_NATIVE))
    params = qpolicy.load(str(dev))
    if params is not None:
        fast = rrf.make_opts(sketch_prec=rrf.SKETCH_BF16, q_policy=rrf.Q_LEARNED, mlp_params=params, steps=steps)
        fms, r_fast, st = timed(fast)
        qs = rrf.opts_q_used(fast)[: steps - 1]
        res["learned_q_bf16_sketch"] = {
            "ms": round(fms, 1), "speedup_vs_plain_fp64_q2": round(pms / fms, 3), "plain_fp64_q2_ms": round(pms, 1),
            "on_target": on_target(r_fast), "plain_on_target": on_target(r_plain), "boundaries": len(ks),
            "max_ratio": max(r_fast.values()), "plain_max_ratio": max(r_plain.values()),
            "q_used": {"mean": round(sum(qs) / len(qs), 3), "hist": [qs.count(v) for v in range(4)]},
            "device_status": st}
    # randUTV_basic with q = 10: e_k <= 1.1 sigma_{k+1} at every block boundary of this matrix (q = 5 .. 8 miss
    # the plateau edge k = n/2 by up to 5 %), against the same method with every product on the DFMA pipe
    qq = 10
    qms, r_q, st = timed(rrf.make_opts(), q=qq)
    qpms, r_qp, _ = timed(rrf.make_opts(gemm_mode=rrf.GEMM_NATIVE), q=qq)
    res["basic_q10"] = {
        "ms": round(qms, 1), "speedup_vs_plain_fp64_same_q": round(qpms / qms, 3), "plain_fp64_ms": round(qpms, 1),
        "on_target": on_target(r_q), "plain_on_target": on_target(r_qp), "boundaries": len(ks),
        "max_ratio": max(r_q.values()), "device_status": st}
    # randUTV_boosted with q = 5, p = b: the oracle meets e_k <= 1.1 sigma_{k+1} at every block boundary of
    # this spectrum's shape with it (2048^2 proxy with the same decay per block), q = 2 at 57 of 63
    qb = 5
    bms, r_boost, st = timed(rrf.make_opts(oversample=b), q=qb)
    bpms, r_bplain, _ = timed(rrf.make_opts(oversample=b, gemm_mode=rrf.GEMM_NATIVE), q=qb)
    res["boosted_q5_p128"] = {
        "ms": round(bms, 1), "speedup_vs_plain_fp64_boosted": round(bpms / bms, 3), "plain_fp64_boosted_ms": round(bpms, 1),
        "speedup_vs_plain_fp64_basic_q2": round(pms / bms, 3), "plain_fp64_boosted_on_target": on_target(r_bplain),
        "on_target": on_target(r_boost), "boundaries": len(ks), "max_ratio": max(r_boost.values()),
        "device_status": st}
    return res


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2106_13402_gb300 import rrf, testmats

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    __graft_entry__.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    n, b, q = args.n, args.b, args.q
    A, s = testmats.make_matrix(n, n, "c2", 11, 12, device=str(dev))
    torch.cuda.synchronize()
    outs = {name: (rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev))
            for name in ("randutv", "powerurv")}
    stream = torch.cuda.current_stream()

    methods = [x for x in args.methods.split(",") if x]
    gemm_mode = {"auto": rrf.GEMM_AUTO, "native": rrf.GEMM_NATIVE, "emulated": rrf.GEMM_EMULATED}[args.gemm]
    opts = rrf.make_opts(gemm_mode=gemm_mode)
    wss = {"randutv": rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, opts), dev),
           "powerurv": rrf.workspace(rrf.powerurv_workspace_bytes(n, n, b, opts), dev)}

    def step():
        if "randutv" in methods:
            rrf.randutv(A, b, q, seed=17, opts=opts, out=outs["randutv"], ws=wss["randutv"], check_status=False)
        if "powerurv" in methods:
            rrf.powerurv(A, b, q, seed=17, opts=opts, out=outs["powerurv"], ws=wss["powerurv"], check_status=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for name in methods:
        st = rrf.lib().rrf_workspace_status(rrf._vp(wss[name].data_ptr()), rrf._stream(None))
        if st != 0:
            raise RuntimeError(f"{name}: device status {st}")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # Timed region: K steps, nothing else enqueued (no profiler events).
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    l0 = rrf.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    launches = rrf.launch_count() - l0
    clocks = sampler.stop()
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    flops = (testmats.flops_randutv(n, n, b, q) if "randutv" in methods else 0.0) + \
        (testmats.flops_powerurv(n, n, q) if "powerurv" in methods else 0.0)
    value = replica_rate(len(methods), world, ms)

    # Profiled pass: the same step with CUDA events around every GEMM and panel launch on its stream, for the
    # dominant kernel's roofline; its step time is reported beside the headline's.
    prof_steps = max(1, min(args.steps, 3))
    rrf.gemm_profile_begin(200000)
    pms_step = _event_ms(torch, lambda: [step() for _ in range(prof_steps)], stream) / prof_steps
    peaks, peak_src = measured_peaks()
    roof = dominant_kernel_roofline(rrf, pms_step, prof_steps, peaks, peak_src)
    roof["measured_over"] = (f"a profiled pass of {prof_steps} steps after the timed region "
                             f"({pms_step:.1f} ms per step with the event profiler on, {ms:.1f} without)")

    # Per-method device times (one more run each, outside the timed region).
    per = {}
    for name in ([] if args.no_per_method else methods):
        f = testmats.flops_randutv(n, n, b, q) if name == "randutv" else testmats.flops_powerurv(n, n, q)
        t = _event_ms(torch, lambda: getattr(rrf, name)(A, b, q, seed=17, opts=opts, out=outs[name], ws=wss[name],
                                                        check_status=False), stream)
        per[name] = {"ms": round(t, 1), "tflops": round(f / t / 1e9, 4), "gflop": round(f / 1e9, 1)}

    # The plain FP64 method (every product on the DFMA pipe) on the same GPU, --plain-reps runs per method.
    plain = None
    if not args.no_plain and args.gemm != "native":
        popts = rrf.make_opts(gemm_mode=rrf.GEMM_NATIVE)
        pper = {}
        for name in methods:
            pws = rrf.workspace((rrf.randutv_workspace_bytes if name == "randutv" else rrf.powerurv_workspace_bytes)(
                n, n, b, popts), dev)
            runs = [_event_ms(torch, lambda: getattr(rrf, name)(A, b, q, seed=17, opts=popts, out=outs[name], ws=pws,
                                                                 check_status=False), stream)
                    for _ in range(max(1, args.plain_reps))]
            pper[name] = {"median_ms": round(statistics.median(runs), 1), "runs_ms": [round(x, 1) for x in runs]}
            del pws
        pms = sum(v["median_ms"] for v in pper.values())
        plain = {"gemm": "native (DFMA)", "ms_per_step": round(pms, 1), "value": round(len(methods) / (pms / 1e3), 5),
                 "per_method": pper, "speedup_of_value": round((len(methods) / (ms / 1e3)) / (len(methods) / (pms / 1e3)), 3)}
        # restore the default path's outputs for the accuracy check below
        for name in methods:
            getattr(rrf, name)(A, b, q, seed=17, opts=opts, out=outs[name], ws=wss[name], check_status=False)
        torch.cuda.synchronize()

    # End to end through the host-buffer C ABI entry points (pinned host memory, copies timed).
    e2e = None
    if not args.no_e2e:
        def pinned(rows, cols):
            return torch.empty((cols, rows), dtype=torch.float64, pin_memory=True).numpy().T
        Ah = pinned(n, n)
        Ah[...] = A.cpu().numpy()
        hout = {name: (pinned(n, n), pinned(n, n), pinned(n, n)) for name in ("randutv", "powerurv")}
        rrf.randutv_host(Ah, b, q, 17, opts=opts, out=hout["randutv"])   # warm-up of the allocator path
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            rrf.randutv_host(Ah, b, q, 17, opts=opts, out=hout["randutv"])
            rrf.powerurv_host(Ah, b, q, 17, opts=opts, out=hout["powerurv"])
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
        e2e = {"value": round(replica_rate(2, world, e2e_s * 1e3), 5), "unit": "factorizations/s",
               "h2d_bytes_per_step": 2 * 8 * n * n, "d2h_bytes_per_step": 2 * 3 * 8 * n * n,
               "s_per_step": round(e2e_s, 3)}

    accuracy = None
    if not args.no_accuracy:
        U, T, V = outs["randutv"]
        res = float(torch.linalg.norm(A - U @ T @ V.t()) / torch.linalg.norm(A))
        eye = torch.eye(n, device=dev, dtype=torch.float64)
        orth_u = float((U.t() @ U - eye).abs().max())
        orth_v = float((V.t() @ V - eye).abs().max())
        lower_zero = bool((torch.tril(T, -1) == 0).all())
        ratios = _boundary_ratios(torch, T, s, b, list(range(b, n, b)))   # every block boundary
        accuracy = {"randutv_residual": res, "randutv_orth_u": orth_u, "randutv_orth_v": orth_v,
                    "t_lower_exact_zero": lower_zero, "e_k_over_sigma_k+1": ratios,
                    "max_ratio": max(ratios.values()) if ratios else None, "boundaries": len(ratios),
                    "on_target": sum(1 for v in ratios.values() if v <= 1.1)}

    extras = None
    if not args.no_extras and world == 1 and n == 8192 and b == 128:
        del wss
        extras = extras_8192(torch, rrf, testmats, A, s, dev, n, b)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(np.asfortranarray(A.cpu().numpy()), n, b, q, args.cpu_pow_n)

    line = {
        "metric": METRIC, "value": round(value, 5), "unit": "factorizations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_c2(n, b, q, methods, args.gemm, world),
        "tflops": round(world * flops / (ms / 1e3) / 1e12, 4),
        "per_method": per,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": round(launches / args.steps, 1),
        "roofline": roof,
        "plain_fp64": plain,
        "accuracy": accuracy,
        "target_configs": extras,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def config_c2(n, b, q, methods, gemm, world):
    """The workload description both arms print (identical for the same arguments)."""
    return {"workload": WORKLOAD, "m": n, "n": n, "b": b, "q": q, "methods": methods, "gemm": gemm,
            "seeds": {"Q1": 11, "Q2": 12, "G": 17}, "l2": "inputs larger than L2 (A is 512 MB)",
            "parallelism": f"replicas x{world}"}


# ------------------------------------------------------------------------------------ reference arm --
def run_reference(args):
    """The oracle (the plain FP64 CPU implementation of the method, as it stands) on the host cores.  Each
    step is a bounded sample of the workload: randUTV's first block step on the same 8192^2 matrix, timed
    through the oracle's entry point (the same work the first step of our randUTV does).  powerURV is timed
    once, in full, on a --cpu-pow-n matrix of the same recipe.  value extrapolates the measured rates to one
    randUTV + powerURV step of the full workload by the flop model; ms_per_step is the measured wall time
    of one sample step."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2106_13402_gb300 import testmats

    oracle.build()
    n, b, q = args.n, args.b, args.q
    A, s = testmats.make_matrix(n, n, "c2", 11, 12, device="cpu") if n <= 4096 else (None, None)
    if A is None:
        import torch
        if torch.cuda.is_available():
            A_t, s = testmats.make_matrix(n, n, "c2", 11, 12, device="cuda")
            A = np.asfortranarray(A_t.cpu().numpy())
            del A_t
        else:
            A, s = testmats.make_matrix(n, n, "c2", 11, 12, device="cpu")
    # warm-up: the oracle's thread pool and pages, on a small matrix (untimed)
    Aw, _ = testmats.make_matrix(256, 256, "c2", 11, 12, device="cpu")
    for _ in range(args.warmup):
        oracle.randutv(Aw, b, q, seed=17, max_steps=1)
    pow_r = cpu_rates(A, n, b, q, args.cpu_pow_n)   # also gives powerURV's rate (timed once)
    samples = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        samples.append(cpu_rates(A, n, b, q, args.cpu_pow_n, pow_rate=pow_r["powerurv_rate"]))
    wall = time.perf_counter() - t_all
    rate = statistics.mean(x["randutv_rate"] for x in samples)
    r = dict(samples[-1], randutv_rate=rate, powerurv_rate=pow_r["powerurv_rate"], powerurv_s=pow_r["powerurv_s"],
             powerurv_gflop=pow_r["powerurv_gflop"])
    per_step_s = cpu_extrapolate(r, n, b, q)
    value = 2.0 / per_step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 7), "unit": "factorizations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall / args.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_c2(n, b, q, ["randutv", "powerurv"], "auto", world),
        "extrapolated": True,
        "sample_steps_run": args.steps,
        "extrapolated_s_per_workload_step": round(per_step_s, 1),
        "powerurv_calibration_s": round(pow_r["powerurv_s"], 2),
        "cpu_baseline": {"value": round(value, 7), "unit": "factorizations/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": "each step: " + cpu_sample_text(r, n, b, q, args.cpu_pow_n)},
        "e2e": {"value": round(value, 7), "unit": "factorizations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------ the other configurations --
def _setup_single_gpu(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch, torch.device("cuda", 0)


def _timed(torch, fn, reps):
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _boundary_ratios(torch, T, s, b, ks):
    return {str(k): round(power_norm(torch, T[k:, k:]) / float(s[k]), 5) for k in ks}


def run_c3_c5(args):
    """c3: randUTV 16384^2, s_j = 1/(1+j), b = 256, q = 2 with the sketch products in BF16 (FP32 accumulate;
    panel QR, Jacobi and WY updates FP64) against the plain FP64 method on the same GPU; e_k / sigma_{k+1} of
    both at sampled boundaries.  c5: randUTV 8192^2 (the 8192^2 spectrum), b = 128, learned per-step q with the
    BF16 sketch against plain FP64 with fixed q = 2; e_k <= 1.1 sigma_{k+1} checked at every boundary."""
    torch, dev = _setup_single_gpu(args)
    from paper_2106_13402_gb300 import qpolicy, rrf, testmats
    c3 = args.workload == "c3"
    n, b = (16384, 256) if c3 else (8192, 128)
    q = 2
    A, s = testmats.make_matrix(n, n, "poly" if c3 else "c2", 21 if c3 else 11, 22 if c3 else 12, device=str(dev))
    steps = n // b
    params = None if c3 else qpolicy.load(str(dev))
    if not c3 and params is None:
        print(json.dumps({"workload": "c5", "unavailable": "no trained policy packaged"}))
        return
    fast = rrf.make_opts(sketch_prec=rrf.SKETCH_BF16, q_policy=rrf.Q_FIXED if c3 else rrf.Q_LEARNED,
                         mlp_params=params, steps=0 if c3 else steps)
    # c5 also times the learned policy with the FP64 sketch (products emulated on the tensor cores)
    fast64 = None if c3 else rrf.make_opts(q_policy=rrf.Q_LEARNED, mlp_params=params, steps=steps)
    plain = rrf.make_opts(gemm_mode=rrf.GEMM_NATIVE)
    out = (rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev))
    ws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, fast), dev)
    for _ in range(args.warmup):
        rrf.randutv(A, b, q, 17, opts=fast, ws=ws, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    l0 = rrf.launch_count()
    rrf.gemm_profile_begin(200000)
    ms = _timed(torch, lambda: rrf.randutv(A, b, q, 17, opts=fast, ws=ws, out=out, check_status=False), args.steps)
    rrf.gemm_profile_end()
    emu_ms, emu_flops, emu_tflops, emu_launches = rrf.gemm_profile_emulated()
    bf_ms, bf_flops, bf_bytes, bf_launches = rrf.gemm_profile_bf16()
    launches = rrf.launch_count() - l0
    clocks = sampler.stop()
    st = rrf.lib().rrf_workspace_status(rrf._vp(ws.data_ptr()), rrf._stream(None))
    qs = rrf.opts_q_used(fast)[: steps - 1] if not c3 else [q] * (steps - 1)
    U, T, V = out
    res = float(torch.linalg.norm(A - U @ T @ V.t()) / torch.linalg.norm(A))
    ks = list(range(b, n, b)) if not c3 else [b, 16 * b, n // 2, n - 2 * b]
    r_fast = _boundary_ratios(torch, T, s, b, ks)
    del ws
    learned64 = None
    if fast64 is not None:
        ws64 = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, fast64), dev)
        rrf.randutv(A, b, q, 17, opts=fast64, ws=ws64, out=out)
        ms64 = _timed(torch, lambda: rrf.randutv(A, b, q, 17, opts=fast64, ws=ws64, out=out, check_status=False),
                      args.steps)
        q64 = rrf.opts_q_used(fast64)[: steps - 1]
        r64 = _boundary_ratios(torch, out[1], s, b, ks)
        learned64 = {"ms": round(ms64, 1), "value": round(1e3 / ms64, 5),
                     "q_used": {"mean": round(sum(q64) / len(q64), 3), "hist": [q64.count(v) for v in range(4)]},
                     "on_target": sum(1 for v in r64.values() if v <= 1.1)}
        del ws64
    # plain FP64 (DFMA products, FP64 sketch, fixed q = 2): one timed run
    pws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, plain), dev)
    rrf.randutv(A, b, q, 17, opts=plain, ws=pws, out=out)
    pms = _timed(torch, lambda: rrf.randutv(A, b, q, 17, opts=plain, ws=pws, out=out, check_status=False), 1)
    r_plain = _boundary_ratios(torch, out[1], s, b, ks)
    del pws
    if learned64 is not None:
        learned64["speedup_vs_plain"] = round(pms / learned64["ms"], 3)
        learned64["worst_ratio_over_plain"] = round(max(r64[k] / r_plain[k] for k in r64), 4)
    flops = testmats.flops_randutv(n, n, b, q)
    peaks, peak_src = measured_peaks()
    peak = float(peaks["bf16_tflops_sustained"])
    ach = emu_tflops / (emu_ms / 1e3) / 1e12 if emu_ms > 0 else 0.0
    on_target = lambda r: sum(1 for v in r.values() if v <= 1.1)
    line = {
        "metric": ("factorizations/s (randUTV, BF16 sketch, 16384^2, b=256, q=2) vs plain FP64" if c3 else
                   "factorizations/s (randUTV, learned q + BF16 sketch, 8192^2, b=128) vs plain FP64 q=2"),
        "value": round(1e3 / ms, 5), "unit": "factorizations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (sketch products bf16 x bf16 -> fp32)", "data": "synthetic",
        "config": {"workload": ("randUTV 16384x16384 A = Q1 diag(1/(1+j)) Q2^T, BF16 sketch" if c3 else
                                "randUTV 8192x8192 A = Q1 diag(s) Q2^T (s_j = 10^(-8j/n), j < n/2, then 1e-4), "
                                "learned q + BF16 sketch"), "m": n, "n": n, "b": b, "q": q,
                   "l2": "inputs larger than L2"},
        "tflops_model": round(flops / (ms / 1e3) / 1e12, 3),
        "plain_fp64": {"ms": round(pms, 1), "value": round(1e3 / pms, 5), "speedup": round(pms / ms, 3),
                       "e_k_over_sigma_k+1": r_plain if c3 else None, "on_target": on_target(r_plain)},
        "e_k_over_sigma_k+1": r_fast if c3 else None,
        "on_target": on_target(r_fast), "boundaries": len(ks),
        "worst_ratio_fast_over_plain": round(max(r_fast[k] / r_plain[k] for k in r_fast), 4),
        "q_used": None if c3 else {"mean": round(sum(qs) / len(qs), 3), "hist": [qs.count(v) for v in range(4)]},
        "learned_fp64_sketch": learned64,
        "residual": res, "device_status": int(st), "clocks": clocks, "gpu_launches": int(launches),
        "roofline": {"kernel": "ozaki_gemm_kernel", "bound": "tensor", "achieved": round(ach, 2), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": None,
                     "peak_source": f"{peak_src} bf16_tflops_sustained", "share_of_step": round(emu_ms / (ms * args.steps), 4),
                     "launches": int(emu_launches)},
        # the BF16 sketch GEMM (tcgen05): HBM-bound skinny products, algorithmic bytes over its event time
        "sketch_roofline": ({"kernel": "tc_gemm_kernel", "bound": "hbm",
                             "achieved": round(bf_bytes / (bf_ms / 1e3) / 1e9, 1), "peak": float(peaks["hbm_gbs"]),
                             "unit": "GB/s", "frac": round(bf_bytes / (bf_ms / 1e3) / 1e9 / float(peaks["hbm_gbs"]), 4),
                             "traffic": None, "tflops": round(bf_flops / (bf_ms / 1e3) / 1e12, 2),
                             "share_of_step": round(bf_ms / (ms * args.steps), 4), "launches": int(bf_launches)}
                            if bf_ms > 0 else None),
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def run_boosted(args):
    """randUTV_boosted (Algorithm 2) on the 8192^2 spectrum: 8192^2, b = 128, q = --boost-q (default 5),
    p = --oversample (default b), the paper's remedy for e_k above 1.1 sigma_{k+1} at block boundaries.  Timed against randUTV_basic with
    the same q and routing and against the plain FP64 method (DFMA products) of the same boosted algorithm;
    e_k / sigma_{k+1} at every block boundary for each."""
    torch, dev = _setup_single_gpu(args)
    from paper_2106_13402_gb300 import rrf, testmats
    n, b, q, p = 8192, 128, args.boost_q, args.oversample
    A, s = testmats.make_matrix(n, n, "c2", 11, 12, device=str(dev))
    fast = rrf.make_opts(oversample=p)
    basic = rrf.make_opts()
    plain = rrf.make_opts(oversample=p, gemm_mode=rrf.GEMM_NATIVE)
    out = (rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev), rrf.fortran_empty(n, n, dev))
    ks = list(range(b, n, b))
    ws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, fast), dev)
    for _ in range(args.warmup):
        rrf.randutv(A, b, q, 17, opts=fast, ws=ws, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    l0 = rrf.launch_count()
    rrf.gemm_profile_begin(200000)
    ms = _timed(torch, lambda: rrf.randutv(A, b, q, 17, opts=fast, ws=ws, out=out, check_status=False), args.steps)
    rrf.gemm_profile_end()
    emu_ms, emu_flops, emu_tflops, emu_launches = rrf.gemm_profile_emulated()
    launches = rrf.launch_count() - l0
    clocks = sampler.stop()
    st = rrf.lib().rrf_workspace_status(rrf._vp(ws.data_ptr()), rrf._stream(None))
    U, T, V = out
    res = float(torch.linalg.norm(A - U @ T @ V.t()) / torch.linalg.norm(A))
    r_fast = _boundary_ratios(torch, T, s, b, ks)
    del ws
    # randUTV_basic, same q and routing
    bws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, basic), dev)
    rrf.randutv(A, b, q, 17, opts=basic, ws=bws, out=out)
    bms = _timed(torch, lambda: rrf.randutv(A, b, q, 17, opts=basic, ws=bws, out=out, check_status=False), args.steps)
    r_basic = _boundary_ratios(torch, out[1], s, b, ks)
    del bws
    # the plain FP64 method: the same boosted algorithm with DFMA products, one timed run
    pws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b, plain), dev)
    rrf.randutv(A, b, q, 17, opts=plain, ws=pws, out=out)
    pms = _timed(torch, lambda: rrf.randutv(A, b, q, 17, opts=plain, ws=pws, out=out, check_status=False), 1)
    r_plain = _boundary_ratios(torch, out[1], s, b, ks)
    del pws
    peaks, peak_src = measured_peaks()
    peak = float(peaks["bf16_tflops_sustained"])
    ach = emu_tflops / (emu_ms / 1e3) / 1e12 if emu_ms > 0 else 0.0
    on_target = lambda r: sum(1 for v in r.values() if v <= 1.1)
    line = {
        "metric": f"factorizations/s (randUTV_boosted, 8192^2, b=128, q={q}, p={p}) vs plain FP64",
        "value": round(1e3 / ms, 5), "unit": "factorizations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "randUTV_boosted 8192x8192 A = Q1 diag(s) Q2^T (s_j = 10^(-8j/n), j < n/2, then "
                               "1e-4)", "m": n, "n": n, "b": b, "q": q, "p": p, "l2": "inputs larger than L2"},
        "plain_fp64": {"ms": round(pms, 1), "value": round(1e3 / pms, 5), "speedup": round(pms / ms, 3),
                       "max_ratio": max(r_plain.values()), "on_target": on_target(r_plain)},
        "basic_same_q": {"ms": round(bms, 1), "max_ratio": max(r_basic.values()), "on_target": on_target(r_basic)},
        "max_ratio": max(r_fast.values()), "on_target": on_target(r_fast), "boundaries": len(ks),
        "e_k_over_sigma_k+1": r_fast,
        "residual": res, "device_status": int(st), "clocks": clocks, "gpu_launches": int(launches),
        "roofline": {"kernel": "ozaki_gemm_kernel", "bound": "tensor", "achieved": round(ach, 2), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": None,
                     "peak_source": f"{peak_src} bf16_tflops_sustained",
                     "share_of_step": round(emu_ms / (ms * args.steps), 4), "launches": int(emu_launches)},
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def run_c4(args):
    """512 FP32 powerURV factorizations (q = 1) of uneven shape, m ~ U[256, 2048], n ~ U[128, m], mixed decays,
    in one CUDA graph of persistent batched kernels with autotuned tiles."""
    torch, dev = _setup_single_gpu(args)
    from paper_2106_13402_gb300 import rrf, testmats
    shapes = testmats.batch_shapes(512, 31)
    plan = rrf.BatchPlan(shapes, b=64, q=1)
    ws = rrf.workspace(plan.workspace_bytes(), dev)
    profs = ("exp8", "poly", "step")
    As = [rrf.as_fortran(testmats.make_matrix(m, n, profs[i % 3], 10000 + i, 20000 + i, device=str(dev))[0].float())
          for i, (m, n) in enumerate(shapes)]
    out = plan.allocate(str(dev))
    t0 = time.perf_counter()
    plan.run(As, out, 31, ws)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        plan.run(As, out, 31, ws)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    l0 = rrf.launch_count()
    ms = _timed(torch, lambda: plan.run(As, out, 31, ws), args.steps)
    launches = rrf.launch_count() - l0
    clocks = sampler.stop()
    fl = sum(testmats.flops_powerurv(m, n, 1) for m, n in shapes)
    worst = 0.0
    for i in range(0, 512, 37):
        U, T, V = out[0][i], out[1][i], out[2][i]
        A = As[i]
        worst = max(worst, float(torch.linalg.norm(A - U @ T @ V.t()) / torch.linalg.norm(A)))
    fp32_peak = 152 * 128 * 2 * 2.070e9 / 1e12
    line = {
        "metric": "factorizations/s (512 uneven FP32 powerURV q=1, one CUDA graph)", "value": round(512 / (ms / 1e3), 2),
        "unit": "factorizations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch of 512: m ~ U[256, 2048], n ~ U[128, m] (seed 31), exp/poly/step decays", "b": 64,
                   "q": 1, "tiles": list(plan.tiles()), "l2": "inputs 1.5 GB, larger than L2"},
        "tflops_model": round(fl / (ms / 1e3) / 1e12, 3), "first_run_s_autotune_capture": round(first_s, 2),
        "worst_sampled_residual": worst, "clocks": clocks, "gpu_launches": int(launches),
        "roofline": {"kernel": "batched FP32 step (whole graph)", "bound": "alu",
                     "achieved": round(fl / (ms / 1e3) / 1e12, 3), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                     "frac": round(fl / (ms / 1e3) / 1e12 / fp32_peak, 4), "traffic": None,
                     "peak_source": "152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz"},
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def run_gemm(args):
    """The emulated FP64 GEMM alone, C = A B with A, B 4096 x 4096 Gaussian (through rrf_gemm_emulated)."""
    torch, dev = _setup_single_gpu(args)
    from paper_2106_13402_gb300 import rrf
    L = rrf.lib()
    m = n = k = 4096
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    A = rrf.as_fortran(torch.randn(m, k, dtype=torch.float64, device=dev, generator=g))
    B = rrf.as_fortran(torch.randn(k, n, dtype=torch.float64, device=dev, generator=g))
    C = rrf.fortran_empty(m, n, dev)
    ws = rrf.workspace(L.rrf_gemm_emulated_workspace(m, n, k), dev)

    def call():
        st = L.rrf_gemm_emulated(b"N", b"N", m, n, k, 1.0, rrf._vp(A.data_ptr()), rrf._ld(A), rrf._vp(B.data_ptr()),
                                 rrf._ld(B), 0.0, rrf._vp(C.data_ptr()), rrf._ld(C), rrf._vp(ws.data_ptr()), ws.numel(),
                                 rrf._stream(None))
        if st != 0:
            raise RuntimeError(f"rrf_gemm_emulated: status {st}")
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    rrf.gemm_profile_begin(1000)
    ms = _timed(torch, call, args.steps)
    rrf.gemm_profile_end()
    emu_ms, emu_flops, emu_tflops, emu_launches = rrf.gemm_profile_emulated()
    clocks = sampler.stop()
    if L.rrf_workspace_status(rrf._vp(ws.data_ptr()), rrf._stream(None)) != 0:
        raise RuntimeError("device status")
    peaks, peak_src = measured_peaks()
    peak = float(peaks["bf16_tflops"])  # a kernel timed alone: the burst figure
    ach = emu_tflops / (emu_ms / 1e3) / 1e12
    fl = 2.0 * m * n * k
    line = {
        "metric": "TFLOP/s (FP64 GEMM 4096^3, emulated on the BF16 tensor cores)", "value": round(fl / (ms / 1e3) / 1e12, 3),
        "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (bf16 digit products, int64 accumulation)",
        "data": "synthetic", "config": {"workload": "C = A B, A and B 4096 x 4096 N(0,1) FP64", "l2": "inputs 256 MB, larger than L2"},
        "clocks": clocks, "gpu_launches": None,
        "roofline": {"kernel": "ozaki_gemm_kernel", "bound": "tensor", "achieved": round(ach, 2), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": kernel_traffic("ozaki_gemm_4096")[0],
                     "traffic_source": kernel_traffic("ozaki_gemm_4096")[1],
                     "traffic_unit": "bytes per launch (dram read + write, ncu)",
                     "algorithmic_bytes": 2 * 7 * m * k * 2 + 8 * m * n,
                     "peak_source": f"{peak_src} bf16_tflops (burst)", "avg_launch_ms": round(emu_ms / max(emu_launches, 1), 4),
                     "share_of_step": round(emu_ms / (ms * args.steps), 4)},
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("c3", "c5"):
        run_c3_c5(args)
    elif args.workload == "c4":
        run_c4(args)
    elif args.workload == "gemm":
        run_gemm(args)
    elif args.workload == "boosted":
        run_boosted(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
