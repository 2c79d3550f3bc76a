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
    p.add_argument("--cpu-sample-steps", type=int, default=2, help="randUTV steps the oracle runs per sample")
    p.add_argument("--methods", default="randutv,powerurv", help="comma list (profiling runs may time one)")
    return p.parse_args()


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
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names[1:], parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
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


def step_flops(n, b, q):
    from paper_2106_13402_gb300 import testmats
    return testmats.flops_randutv(n, n, b, q) + testmats.flops_powerurv(n, n, q)


def cpu_sample(A_np, n, b, q, sample_steps):
    """Time the oracle (as it stands) on the first `sample_steps` randUTV steps of the same matrix and
    extrapolate its flop rate to one full step (randUTV + powerURV) by the flop model."""
    import oracle
    from paper_2106_13402_gb300 import testmats

    sample_flops = testmats.flops_randutv(n, n, b, q, max_steps=sample_steps)
    t0 = time.perf_counter()
    oracle.randutv(A_np, b, q, seed=17, max_steps=sample_steps)
    dt = time.perf_counter() - t0
    rate = sample_flops / dt
    per_step_s = step_flops(n, b, q) / rate
    return {"value": 2.0 / per_step_s, "unit": "factorizations/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": (f"first {sample_steps} of {n // b} randUTV steps of the same {n}x{n} matrix "
                       f"({sample_flops / 1e9:.0f} GFLOP in {dt:.1f} s, {rate / 1e9:.2f} GFLOP/s), "
                       f"extrapolated to one randUTV + powerURV step by the flop model"),
            "seconds": dt}


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
    wss = {"randutv": rrf.workspace(rrf.randutv_workspace_bytes(n, n, b), dev),
           "powerurv": rrf.workspace(rrf.powerurv_workspace_bytes(n, n, b), dev)}
    stream = torch.cuda.current_stream()

    methods = [x for x in args.methods.split(",") if x]

    def step():
        if "randutv" in methods:
            rrf.randutv(A, b, q, seed=17, out=outs["randutv"], ws=wss["randutv"], check_status=False)
        if "powerurv" in methods:
            rrf.powerurv(A, b, q, seed=17, out=outs["powerurv"], ws=wss["powerurv"], check_status=False)

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

    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    l0 = rrf.launch_count()
    rrf.gemm_profile_begin(200000)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    gemm_ms, gemm_flops, gemm_launches = rrf.gemm_profile_end()
    launches = rrf.launch_count() - l0
    clocks = sampler.stop()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    flops = (testmats.flops_randutv(n, n, b, q) if "randutv" in methods else 0.0) + \
        (testmats.flops_powerurv(n, n, q) if "powerurv" in methods else 0.0)
    value = world * len(methods) / (ms / 1e3)

    # Per-method device times (one more run each, outside the timed region).
    per = {}
    for name in methods:
        f = testmats.flops_randutv(n, n, b, q) if name == "randutv" else testmats.flops_powerurv(n, n, q)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        getattr(rrf, name)(A, b, q, seed=17, out=outs[name], ws=wss[name], check_status=False)
        a1.record(stream)
        a1.synchronize()
        t = a0.elapsed_time(a1)
        per[name] = {"ms": round(t, 1), "tflops": round(f / t / 1e9, 4), "gflop": round(f / 1e9, 1)}

    # End to end through the host-buffer C ABI entry points (pinned host memory, copies timed).
    e2e = None
    if not args.no_e2e:
        def pinned(rows, cols):
            return torch.empty((cols, rows), dtype=torch.float64, pin_memory=True).numpy().T
        Ah = pinned(n, n)
        Ah[...] = A.cpu().numpy()
        hout = {name: (pinned(n, n), pinned(n, n), pinned(n, n)) for name in ("randutv", "powerurv")}
        rrf.randutv_host(Ah, b, q, 17, out=hout["randutv"])   # warm-up of the allocator path
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            rrf.randutv_host(Ah, b, q, 17, out=hout["randutv"])
            rrf.powerurv_host(Ah, b, q, 17, out=hout["powerurv"])
        e2e_s = (time.perf_counter() - t0) / args.steps
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": round(world * 2.0 / e2e_s, 5), "unit": "factorizations/s",
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
        ratios = {}
        for k in (b, 16 * b, n // 2, n - 2 * b):
            ratios[str(k)] = round(power_norm(torch, T[k:, k:]) / float(s[k]), 5)
        accuracy = {"randutv_residual": res, "randutv_orth_u": orth_u, "randutv_orth_v": orth_v,
                    "t_lower_exact_zero": lower_zero, "e_k_over_sigma_k+1": ratios}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(np.asfortranarray(A.cpu().numpy()), n, b, q, args.cpu_sample_steps)

    gemm_avg_ms = gemm_ms / max(gemm_launches, 1)
    achieved = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else 0.0
    line = {
        "metric": METRIC, "value": round(value, 5), "unit": "factorizations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": n, "n": n, "b": b, "q": q, "methods": methods,
                   "seeds": {"Q1": 11, "Q2": 12, "G": 17}, "l2": "inputs larger than L2 (A is 512 MB)",
                   "parallelism": f"replicas x{world}"},
        "tflops": round(world * flops / (ms / 1e3) / 1e12, 4),
        "per_method": per,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": round(launches / args.steps, 1),
        "roofline": {"kernel": "gemm_f64_kernel (+ split-K reduction)", "bound": "alu", "achieved": round(achieved, 4),
                     "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                     "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": None,
                     "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe; recipe nominal 1.25)",
                     "launches": int(gemm_launches), "avg_launch_ms": round(gemm_avg_ms, 4),
                     "share_of_step": round(gemm_ms / (ms * args.steps), 4)},
        "accuracy": accuracy,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------------ reference arm --
def run_reference(args):
    """The oracle (plain FP64 CPU implementation of the method), timed on the host cores on a bounded
    sample of the same workload per step."""
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
    samples = []
    for _ in range(args.warmup):
        cpu_sample(A, n, b, q, 1)
    for _ in range(args.steps):
        samples.append(cpu_sample(A, n, b, q, 1))
    per_step_s = statistics.mean(2.0 / x["value"] for x in samples)
    value = 2.0 / per_step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 7), "unit": "factorizations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_step_s * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": n, "n": n, "b": b, "q": q, "methods": ["randutv", "powerurv"],
                   "seeds": {"Q1": 11, "Q2": 12, "G": 17}, "l2": "host run", "parallelism": "host cores"},
        "cpu_baseline": {"value": round(value, 7), "unit": "factorizations/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": samples[-1]["sample"]},
        "e2e": {"value": round(value, 7), "unit": "factorizations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
