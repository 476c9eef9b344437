"""Benchmark of the integer matrix power A^n on GB300 through libmatpow.

Default workload (one "step"): a single N=512 float32 matrix with entries
N(0, 1/N), seed 0, raised to every power n in {2, 16, 128, 1024} by binary
square-and-multiply -- G(n) = {1, 4, 7, 10} products, 22 in all.  The metric
is effective TFLOP/s = sum over the step of G(n) * 2 N^3 / time (the
algorithmic count: the three bfloat16 products of the split path and the
n-1 products of the naive method are not counted).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

L2_FLUSH_BYTES = 256 << 20  # > 129 MB of L2

WORKLOADS = {
    "single512": dict(N=512, ns=[2, 16, 128, 1024], gen="gaussian",
                      desc="single N=512 N(0,1/N) float32, n in {2,16,128,1024}, seed 0"),
    "stoch64": dict(N=64, ns=[100], gen="stochastic",
                    desc="single N=64 exact row-stochastic float32, n=100, seed 0"),
    "large8192": dict(N=8192, ns=[2 ** 20], gen="stochastic",
                      desc="single N=8192 exact row-stochastic float32, n=2^20, seed 0"),
    # one product at N=4096 (operands 64 MB each, beyond L2): profiling case
    "probe4096": dict(N=4096, ns=[2], gen="stochastic",
                      desc="single N=4096 exact row-stochastic float32, n=2 (one product), seed 0"),
}


def gemm_count(n: int) -> int:
    return 0 if n <= 1 else (n.bit_length() - 1) + bin(n).count("1") - 1


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_input(wk):
    from paper_1204_3052_gb300 import workloads as wl
    if wk["gen"] == "gaussian":
        return wl.gaussian(wk["N"], 0)
    return wl.stochastic_exact(wk["N"], 0)


# ---------------------------------------------------------------------------- oracle timing

def cpu_sample(wk, budget_s: float = 15.0, threads: int = 0):
    """Time the CPU oracle on a bounded sample of the workload (effective TFLOP/s).

    The sample is the workload's list of powers, repeated until about
    ``budget_s`` seconds of oracle time; for large N (where one power takes
    far longer) it is a single product (n = 2) of the same matrix.
    """
    import oracle
    A = make_input(wk)
    N = wk["N"]
    cores = oracle.set_threads(threads)
    per_power_est = max(gemm_count(n) for n in wk["ns"]) * 2.0 * N ** 3 / (1.5e9 * cores)
    ns = sorted(wk["ns"]) if per_power_est < budget_s else [2]
    done_flop, t_total, reps = 0.0, 0.0, 0
    while True:
        for n in ns:
            t0 = time.perf_counter()
            oracle.matpow_f64(A, n)
            t_total += time.perf_counter() - t0
            done_flop += gemm_count(n) * 2.0 * N ** 3
        reps += 1
        if t_total >= budget_s or t_total * (reps + 1) / reps > 2 * budget_s or reps >= 1000:
            break
    return {"value": done_flop / t_total / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": "float64 triple-loop square-and-multiply, N=%d, n in %s x %d (%.1f s)" % (
                N, ns, reps, t_total)}


def run_reference(args, wk, world, rank):
    if rank != 0:
        return
    res = []
    for _ in range(args.warmup):
        pass  # the oracle has nothing to warm up beyond loading
    cb = None
    for _ in range(max(args.steps, 1)):
        cb = cpu_sample(wk, budget_s=args.ref_budget)
        res.append(cb["value"])
    value = statistics.median(res)
    cb["value"] = value
    line = {"metric": "matpow effective TFLOP/s", "value": value, "unit": "TFLOP/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wk["desc"]}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------- GPU timing

def run_ours(args, wk, world, rank, local):
    import torch
    from paper_1204_3052_gb300 import matpow as mpw

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_src = load_peaks()
    N, ns = wk["N"], wk["ns"]
    prec = args.precision
    flop_step = sum(gemm_count(n) for n in ns) * 2.0 * N ** 3

    A_host = make_input(wk)
    A = torch.from_numpy(A_host).to(dev)
    outs = [torch.empty_like(A) for _ in ns]
    lgs = torch.zeros(len(ns), dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    plan = mpw.Plan(N, prec, device=local)

    def step(s):
        for i, n in enumerate(ns):
            st = mpw.matpow_f32(plan.h, A, N, n, outs[i], lgs[i:i + 1], s)
            if st != 0:
                mpw._check(st, plan.h)

    # ---- device-resident timed region
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step(stream)
        plan.check(stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        launches0 = plan.launch_count()
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (not timed)
            evs[k][0].record(stream)
            step(stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        barrier(world)
        clocks = sampler.stop()
        launches = plan.launch_count() - launches0
        st = plan.sync(stream)
        step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = sum(step_ms)
    t_ms = max_over_ranks(world, t_ms, dev)
    value = world * args.steps * flop_step / (t_ms * 1e-3) / 1e12

    # ---- accuracy of this run against the oracle (reported, not timed)
    errs = {}
    if rank == 0 and not args.no_check:
        import oracle
        for i, n in enumerate(ns):
            if N > 1024:
                continue
            M, e, _ = oracle.matpow_f64(A_host, n)
            errs[str(n)] = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lgs[i].item()), M, e)

    # ---- end to end through the C-ABI with host buffers
    A_pin = torch.from_numpy(A_host).pin_memory()
    outs_pin = [torch.empty(A_host.shape, dtype=torch.float32).pin_memory() for _ in ns]
    lg_pin = torch.zeros(len(ns), dtype=torch.int64).pin_memory()
    e2e_steps = max(args.steps, 3)
    with torch.cuda.stream(stream):
        def e2e_step():
            A.copy_(A_pin, non_blocking=True)
            step(stream)
            for i in range(len(ns)):
                outs_pin[i].copy_(outs[i], non_blocking=True)
            lg_pin.copy_(lgs, non_blocking=True)
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(world, e0.elapsed_time(e1), dev)
    e2e_value = world * e2e_steps * flop_step / (e2e_ms * 1e-3) / 1e12

    # ---- dominant kernel: per-launch CUDA-event timing on the launching stream
    plan.set_option(mpw.OPT_TIMING, 1)
    kind = {"fp32": mpw.KERNEL_SIMT, "bf16": mpw.KERNEL_TC, "bf16x3": mpw.KERNEL_TC}[prec]
    if N <= 64:
        kind = mpw.KERNEL_TINY
    with torch.cuda.stream(stream):
        plan.kernel_time(kind, reset=True)
        for _ in range(max(args.steps, 3)):
            flush.zero_()
            step(stream)
        torch.cuda.synchronize()
        kl, kms, kflop = plan.kernel_time(kind, reset=True)
    plan.set_option(mpw.OPT_TIMING, 0)
    products = 3.0 if prec == "bf16x3" else 1.0
    if kind == mpw.KERNEL_TC:
        achieved = kflop * products / (kms * 1e-3) / 1e12
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "tc_gemm", "peak_source": peak_src + " bf16 burst",
                "counted": "%d bfloat16 product(s) per term" % int(products)}
    else:
        # float32 FFMA peak: 152 SMs x 128 lanes x 2 flop x max SM clock
        smax = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * smax * 1e6 / 1e12
        achieved = kflop / (kms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "simt_gemm" if kind == mpw.KERNEL_SIMT else "tiny_chain",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % smax}
    roof["launches_timed"] = kl
    roof["avg_launch_us"] = kms * 1e3 / max(kl, 1)

    if rank != 0:
        return
    cb = cpu_sample(wk, budget_s=args.cpu_budget) if world == 1 and not args.no_cpu else None
    line = {
        "metric": "matpow effective TFLOP/s", "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3"}[prec],
        "data": "synthetic",
        "config": {"workload": wk["desc"], "precision": prec, "gemms_per_step":
                   sum(gemm_count(n) for n in ns), "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "rel_frobenius_vs_f64": errs,
        "status": st,
        "wall_s_timed": wall,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "TFLOP/s",
                "h2d_bytes_per_step": int(A_host.nbytes),
                "d2h_bytes_per_step": int(A_host.nbytes * len(ns) + 8 * len(ns))},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cb,
    }
    print(json.dumps(line))
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="single512")
    ap.add_argument("--precision", choices=["fp32", "bf16", "bf16x3"], default="bf16x3")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--ref-budget", type=float, default=5.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wk = WORKLOADS[args.workload]
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, wk, world, rank)
    else:
        run_ours(args, wk, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
