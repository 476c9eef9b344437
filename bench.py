"""Benchmark of the integer matrix power A^n on GB300 through libmatpow.

Default workload (one "step"): a single N=8192 float32 exactly row-stochastic
matrix (rows U[0,1) normalised so that every float32 row sums to 1 exactly),
seed 0, raised to n = 2^20 by binary square-and-multiply: 20 squarings,
G(n) = 20 products of 2 N^3.  The metric is effective TFLOP/s = G(n) 2 N^3 /
time (the algorithmic count: the three bfloat16 products of the BF16X3 split
and the n-1 products of the naive method are not counted).  The default
precision there is the two-slice exact split (BF16X3), the cheapest
tensor-core path whose error stays within 2e-5 ceil(log2 n) on these inputs;
the error is measured against the closed form 1 pi^T (pi by float64 power
iteration) on 64 sampled rows, beside the largest row-sum deviation.  The
line also carries the plain FP32 SIMT and plain BF16 paths timed on the same
workload, and the N=512 Gaussian workload (n in {2,16,128,1024}) on every
float path with its errors per n.

Other workloads (``--workload``): the N=512 Gaussian powers alone
(``single512``), the 4096-matrix batch, the request server, A^n mod p,
e^A, the naive-method comparison and the N=64 on-chip chain.  ``--api
single`` issues one matpow_f32 call per power for multi-power workloads
(default: one matpow_batched call).

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

# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum +
# dram__bytes_write.sum) from one ncu capture, keyed by (workload, precision);
# the summaries under profiles/ give the command.  Reset to None whenever the
# kernel changes.
TRAFFIC = {
    ("single512", "bf16x6"): (1.15e6, "ncu one-pass dram__bytes_read.sum + dram__bytes_write.sum of "
                                      "tc_chain_split_kernel<64, 3, 2>, one launch per step"),
    ("batched4096", "bf16x6"): (7.73e8, "ncu one-pass dram__bytes_read.sum + dram__bytes_write.sum of "
                                        "tc_fxb_persist_kernel<3> (two epilogue groups, transposed looped stores), average "
                                        "over the 12 level launches of one step"),
    ("modp2048", "bf16x3"): (2.70e7, "ncu one-pass dram__bytes_read.sum + dram__bytes_write.sum of "
                                     "tc_modp_kernel, average over the 14 launches of one step"),
    ("stoch64", "fp32"): (5.66e4, "ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                                  "tiny_cluster_kernel, one launch"),
    ("large8192", "bf16x3"): (3.05e9, "ncu one-pass dram__bytes_read.sum + dram__bytes_write.sum of "
                                      "tc_fxb_kernel<128, 2>, one product at full size"),
}

# bfloat16 tensor-core products per algorithmic product (roofline counting)
# and the arithmetic each precision computes in
PRODUCTS = {"fp32": 1.0, "bf16": 1.0, "bf16x3": 3.0, "bf16x6": 6.0}
DTYPE = {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3", "bf16x6": "bf16x6"}

WORKLOADS = {
    "single512": dict(N=512, ns=[2, 16, 128, 1024], gen="gaussian", prec="bf16x6",
                      desc="single N=512 N(0,1/N) float32, n in {2,16,128,1024}, seed 0"),
    "stoch64": dict(N=64, ns=[100], gen="stochastic", prec="fp32",
                    desc="single N=64 exact row-stochastic float32, n=100, seed 0"),
    "large8192": dict(N=8192, ns=[2 ** 20], gen="stochastic", prec="bf16x3",
                      desc="single N=8192 exact row-stochastic float32, n=2^20, seed 0"),
    "batched4096": dict(kind="batched", count=4096, n_max=4096, N=256, ns=[], prec="bf16x6",
                        desc="batched: 4096 N(0,1/N) float32 matrices, N uniform over {16,...,256}, "
                             "n log-uniform in [1,4096], seed 0; one grouped launch per level"),
    "serving": dict(kind="serving", count=20000, N=2048, ns=[], prec="bf16x6",
                    desc="serving: 20000 Poisson-arrival requests, N log-uniform [8,2048], n log-uniform "
                         "[1,2^30], 90% float / 10% mod 65521, seed 0"),
    "modp2048": dict(kind="modp", N=2048, ns=[1000], p=65521, prec="bf16x3",
                     desc="single N=2048 U{0..65520} uint32, A^1000 mod 65521 (14 products), seed 0"),
    # the paper's comparison (Sec. 5.2): square-and-multiply against the naive
    # GPU method (n - 1 products, one launch each) at its orders and powers
    "vs_naive": dict(kind="naive", Ns=[128, 256, 512], ns_list=[64, 256, 1024], N=512, ns=[],
                     prec="bf16x6", gen="gaussian",
                     desc="N in {128,256,512} N(0,1/N) float32, n in {64,256,1024}, seed 0: "
                          "square-and-multiply vs the naive n-1 product method on the GPU"),
    # the matrix exponential on the same kernels (scaling and squaring)
    "expm512": dict(kind="expm", N=512, scale=4.0, ns=[], prec="bf16x6", gen="gaussian",
                    desc="e^A of a single N=512 4 N(0,1/N) float32 matrix (||A||_1 ~ 70: 7 squarings), seed 0"),
    # a smaller batch of the same mix (profiling case: a few hundred MB on the device)
    "batched512": dict(kind="batched", count=512, n_max=4096, N=256, ns=[], prec="bf16x6",
                       desc="batched: 512 N(0,1/N) float32 matrices, N uniform over {16,...,256}, "
                            "n log-uniform in [1,4096], seed 0; one grouped launch per level"),
    # one product at N=8192 (operand planes 256 MB, twice the L2; ~2 GB on the
    # device in all): the headline kernel's profiling case
    "probe8192": dict(N=8192, ns=[2], gen="stochastic", prec="bf16x3",
                      desc="single N=8192 exact row-stochastic float32, n=2 (one product), seed 0"),
    # one product at N=4096 (operands 64 MB each, beyond L2): profiling case
    "probe4096": dict(N=4096, ns=[2], gen="stochastic", prec="bf16x3",
                      desc="single N=4096 exact row-stochastic float32, n=2 (one product), seed 0"),
}


def tile_table_path(args):
    """The tile table the bench's plans load: the tuned table shipped with the
    package (``--tile-table default``, when present), a file, or none."""
    if args.tile_table == "none":
        return None
    if args.tile_table == "default":
        from paper_1204_3052_gb300 import matpow as mpw
        return mpw.DEFAULT_TILE_TABLE if os.path.exists(mpw.DEFAULT_TILE_TABLE) else None
    return args.tile_table


_FP32_PEAK = {}


def fp32_peak(dev_index: int):
    """Measured FP32 FFMA TFLOP/s of the device (register-only probe of the
    library, best of 5 timed launches of ~0.1 s of work), cached per device;
    with a note of where it came from."""
    if dev_index not in _FP32_PEAK:
        from paper_1204_3052_gb300 import matpow as mpw
        plan = mpw.Plan(64, "fp32", device=dev_index)
        v = mpw.measure_fp32_peak(plan.h, iters=1 << 17)
        plan.close()
        _FP32_PEAK[dev_index] = (v, "measured: matpow_selftest_ffma, 8 CTAs x 256 threads per SM, "
                                    "8 register FFMA chains per thread, best of 5")
    return _FP32_PEAK[dev_index]


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

def cpu_sample(wk, budget_s: float = 15.0, threads: int = 0, A=None):
    """Time the CPU oracle on a bounded sample of the workload (effective TFLOP/s).

    The sample is the workload's list of powers, repeated until about
    ``budget_s`` seconds of oracle time.  Where one power takes far longer
    (large N), it is the leading rows of the power's first product A A, by
    the oracle's triple loop, taken in chunks until about ``budget_s``
    seconds (2 N^2 flop per row).
    """
    import oracle
    if A is None:
        A = make_input(wk)
    N = wk["N"]
    cores = oracle.set_threads(threads)
    per_power_est = max(gemm_count(n) for n in wk["ns"]) * 2.0 * N ** 3 / (1.5e9 * cores)
    if per_power_est >= budget_s:
        A64 = np.ascontiguousarray(A, dtype=np.float64)
        chunk = max(cores, 8)
        rows, t_total = 0, 0.0
        while rows < N and t_total < budget_s:
            r1 = min(N, rows + chunk)
            t0 = time.perf_counter()
            oracle.gemm_rows_f64(A64, A64, rows, r1)
            t_total += time.perf_counter() - t0
            rows = r1
        return {"value": rows * 2.0 * N * N / t_total / 1e12, "unit": "TFLOP/s", "cores": cores,
                "kind": "oracle",
                "sample": "float64 triple loop, rows 0..%d of the first product A A of the N=%d power "
                          "(%.1f s; one whole power is %d such products)" % (
                              rows - 1, N, t_total, max(gemm_count(n) for n in wk["ns"]))}
    ns = sorted(wk["ns"])
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


def cpu_sample_modp(wk, budget_s):
    """Oracle A^64 mod p (6 products) of the workload's leading 512 x 512 block,
    repeated for about budget_s; effective TFLOP/s."""
    import oracle
    from paper_1204_3052_gb300 import workloads as wl
    A = wl.modp_uniform(wk["N"], wk["p"], 0)[:512, :512].copy()
    cores = oracle.set_threads(0)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.matpow_modp(A, 64, wk["p"])
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s or reps >= 100:
            break
    return {"value": reps * 6 * 2.0 * 512 ** 3 / dt / 1e12, "unit": "TFLOP/s", "cores": cores,
            "kind": "oracle", "sample": "uint64 triple-loop A^64 mod p of the leading 512 x 512 block "
                                        "x %d (%.1f s)" % (reps, dt)}


def expm_input(wk):
    from paper_1204_3052_gb300 import workloads as wl
    return (wl.gaussian(wk["N"], 0) * wk["scale"]).astype(np.float32)


def expm_flop(A) -> float:
    """Algorithmic flop of e^A by the library's method: (5 + s) products of
    2N^3 (B^2, B^3, B^4, two Paterson-Stockmeyer products, s squarings)."""
    import oracle
    return (5 + oracle.expm_scaling(A, 1.0)) * 2.0 * A.shape[0] ** 3


def cpu_sample_expm(wk, budget_s):
    """The float64 oracle e^A of the workload's matrix, repeated for about
    budget_s; e^A per second times the library method's algorithmic flop."""
    import oracle
    A = expm_input(wk)
    cores = oracle.set_threads(0)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.expm_f64(A)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s or reps >= 100:
            break
    return {"value": reps * expm_flop(A) / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": "float64 scaling and squaring of the exponential series (triple-loop products), "
                      "N=%d x %d (%.1f s)" % (wk["N"], reps, dt)}


def cpu_sample_list(items, budget_s):
    """Oracle over (A, n, p) items in order until ~budget_s; effective TFLOP/s."""
    import oracle
    cores = oracle.set_threads(0)
    t0 = time.perf_counter()
    done, k = 0.0, 0
    for A, n, p in items:
        if k and time.perf_counter() - t0 >= budget_s:
            break
        if p:
            oracle.matpow_modp(A, n, p)
        else:
            oracle.matpow_f64(A, n)
        done += gemm_count(n) * 2.0 * A.shape[0] ** 3
        k += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "items_per_s": k / dt,
            "sample": "oracle on the first %d items of the workload (%.1f s)" % (k, dt)}


def reference_items(wk):
    from paper_1204_3052_gb300 import workloads as wl
    if wk.get("kind") == "batched":
        bd = wl.batched_draw(count=wk["count"], seed=0, n_max=wk["n_max"])
        for N, n, sd in zip(bd.Ns, bd.ns, bd.seeds):
            yield wl.gaussian(int(N), int(sd)), int(n), 0
    else:
        for r in wl.serving_stream(count=wk["count"], seed=0):
            yield wl.request_matrix(r), r.n, (r.p if r.kind else 0)


def config_for(args, wk, world):
    """The `config` object of a bench line, identical for both arms."""
    from paper_1204_3052_gb300 import workloads as wl
    tt = tile_table_path(args)
    cfg = {"workload": wk["desc"], "precision": args.precision,
           "tile_table": os.path.basename(tt) if tt else "built-in rules"}
    if wk.get("kind") == "batched":
        bd = wl.batched_draw(count=wk["count"], seed=0, n_max=wk["n_max"])
        cfg.update(matrices=wk["count"], gemms_per_step=int(sum(gemm_count(int(n)) for n in bd.ns)),
                   l2="flushed between timed steps (256 MB write)")
    elif wk.get("kind") == "serving":
        cfg.update(requests=wk["count"], load_sweep=list(args.sweep),
                   sweep_requests=min(wk["count"], args.sweep_count) if args.sweep_count > 0 else wk["count"])
    elif wk.get("kind") == "naive":
        cfg.update(orders=wk["Ns"], powers=wk["ns_list"], l2="flushed between timed runs (256 MB write)")
    elif wk.get("kind") == "modp":
        cfg.update(p=wk["p"], gemms_per_step=sum(gemm_count(n) for n in wk["ns"]),
                   l2="flushed between timed steps (256 MB write)")
        cfg["precision"] = "exact mod p (byte-sliced bfloat16 tensor-core products)"
    elif wk.get("kind") == "expm":
        import oracle
        s = oracle.expm_scaling(expm_input(wk), 1.0)
        cfg.update(squarings=s, gemms_per_step=5 + s, l2="flushed between timed steps (256 MB write)",
                   api="matpow_expm")
    else:
        cfg.update(gemms_per_step=sum(gemm_count(n) for n in wk["ns"]),
                   l2="flushed between timed steps (256 MB write)",
                   parallelism="replicas" if world > 1 else "single")
        if args.chain_mode != 1:
            cfg["chain_mode"] = args.chain_mode
        cfg["api"] = ("one matpow_batched call over the %d powers" % len(wk["ns"])
                      if args.api == "batched" and len(wk["ns"]) > 1 else "matpow_f32 per power")
    return cfg


def run_reference(args, wk, world, rank):
    if rank != 0:
        return
    res = []
    walls = []
    cb = None
    A_ref = None
    serving = wk.get("kind") == "serving"
    for _ in range(max(args.steps, 1)):
        t_step = time.perf_counter()
        if wk.get("kind") in ("batched", "serving"):
            cb = cpu_sample_list(reference_items(wk), args.ref_budget)
        elif wk.get("kind") == "modp":
            cb = cpu_sample_modp(wk, args.ref_budget)
        elif wk.get("kind") == "expm":
            cb = cpu_sample_expm(wk, args.ref_budget)
        elif wk.get("kind") == "naive":
            cb = cpu_sample(dict(wk, ns=wk["ns_list"]), budget_s=args.ref_budget)
        else:
            if A_ref is None:
                A_ref = make_input(wk)
            cb = cpu_sample(wk, budget_s=args.ref_budget, A=A_ref)
        res.append(cb["items_per_s"] if serving else cb["value"])
        walls.append(time.perf_counter() - t_step)
    value = statistics.median(res)
    cb["value"] = value
    metric, unit = ("matpow serving req/s", "req/s") if serving else ("matpow effective TFLOP/s", "TFLOP/s")
    cb["unit"] = unit
    line = {"metric": metric, "value": value, "unit": unit,
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(walls) * 1e3,
            "ms_per_step_is": "wall time of one bounded sample of the workload (a step of the oracle)",
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 mod p" if wk.get("kind") == "modp" else "f64",
            "data": "synthetic", "config": config_for(args, wk, world), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------- GPU timing

def stated_tolerance(n: int) -> float:
    """Relative Frobenius bound for float32-class results: 2e-5 * ceil(log2 n)
    (an exact copy, 1e-7, for n = 1)."""
    return 1e-7 if n <= 1 else 2e-5 * math.ceil(math.log2(n))


def errors_of(wk, A_host, ns, outs, lgs):
    """Error of each power against the oracle (float64 square-and-multiply), or
    for large stochastic powers against the closed form 1 pi^T on 64 sampled
    rows plus the largest row-sum deviation; with the stated-error verdict."""
    import oracle
    N = wk["N"]
    errs = {}
    met = True
    for i, n in enumerate(ns):
        Mg = outs[i].cpu().numpy().astype(np.float64)
        lg = int(lgs[i].item())
        if N > 1024:
            if wk["gen"] == "stochastic" and n >= 2 ** 10:
                pi = oracle.stationary(A_host)
                Vg = np.ldexp(Mg, lg)
                rows = np.random.default_rng(0).choice(N, 64, replace=False)
                want = np.tile(pi, (64, 1))
                errs[str(n)] = float(np.linalg.norm(Vg[rows] - want) / np.linalg.norm(want))
                errs["max_rowsum_dev"] = float(np.max(np.abs(Vg.sum(axis=1) - 1.0)))
                met = met and errs[str(n)] <= stated_tolerance(n)
            continue
        M, e, _ = oracle.matpow_f64(A_host, n)
        errs[str(n)] = oracle.rel_frobenius(Mg, lg, M, e)
        met = met and errs[str(n)] <= stated_tolerance(n)
    if errs:
        errs["within_2e-5_ceil_log2_n"] = bool(met)
    return errs


def path_compare(args, wk, A, A_host, flush, stream, value, prec="fp32"):
    """Time another precision's path (plain FP32 SIMT by default, the metric's
    comparator) on the same workload, with the same L2 flush and event
    timing and fewer steps; report its value, errors and the ratio."""
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    N, ns = wk["N"], wk["ns"]
    plan = mpw.Plan(N, prec, device=A.device.index)
    outs = [torch.empty_like(A) for _ in ns]
    lgs = torch.zeros(len(ns), dtype=torch.int64, device=A.device)
    steps = max(1, min(args.steps, 3 if N > 2048 else 10))

    def step():
        for i, n in enumerate(ns):
            st = mpw.matpow_f32(plan.h, A, N, n, outs[i], lgs[i:i + 1], stream)
            if st != 0:
                mpw._check(st, plan.h)

    with torch.cuda.stream(stream):
        flush.zero_()
        step()
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        plan.check(stream)
    flop_step = sum(gemm_count(n) for n in ns) * 2.0 * N ** 3
    v = steps * flop_step / (ms * 1e-3) / 1e12
    errs = {} if args.no_check else errors_of(wk, A_host, ns, outs, lgs)
    plan.close()
    out = {"precision": prec, "value": v, "unit": "TFLOP/s", "steps": steps, "rel_frobenius_vs_f64": errs,
           "ratio_this_path_over_it": value / v if v else None}
    if prec == "fp32":  # the comparator's own quality: its rate against the measured FFMA peak
        pk, _ = fp32_peak(A.device.index)
        out["measured_fp32_peak_tflops"] = pk
        out["frac_of_fp32_peak"] = v / pk
    return out


def config2_table(args, dev, flush, stream):
    """The N = 512 Gaussian workload (powers 2, 16, 128, 1024) on every float
    path -- plain FP32 SIMT, plain BF16, BF16X3 and BF16X6 -- per step one
    matpow_batched call over the four powers (the exact splits and FP32; plain
    BF16 has no grouped launch and takes one matpow_f32 call per power), CUDA
    events, L2 flushed; each power's error against the float64 oracle and
    whether it met 2e-5 ceil(log2 n)."""
    import torch
    import oracle
    from paper_1204_3052_gb300 import matpow as mpw
    wk = WORKLOADS["single512"]
    N, ns = wk["N"], wk["ns"]
    A_host = make_input(wk)
    A = torch.from_numpy(A_host).to(dev)
    ref = {} if args.no_check else {n: oracle.matpow_f64(A_host, n)[:2] for n in ns}
    flop_step = sum(gemm_count(n) for n in ns) * 2.0 * N ** 3
    out_all = torch.empty((len(ns), N, N), dtype=torch.float32, device=dev)
    outs = [out_all[i] for i in range(len(ns))]
    lgs = torch.zeros(len(ns), dtype=torch.int64, device=dev)
    table = {}
    for prec in ("fp32", "bf16", "bf16x3", "bf16x6"):
        plan = mpw.Plan(N, prec, device=dev.index)
        steps = max(3, min(args.steps, 20))

        def step():
            if prec == "bf16":
                for i, n in enumerate(ns):
                    mpw._check(mpw.matpow_f32(plan.h, A, N, n, outs[i], lgs[i:i + 1], stream), plan.h)
            else:
                mpw._check(mpw.matpow_batched(plan.h, [A] * len(ns), [N] * len(ns), ns, outs, lgs, stream),
                           plan.h)

        with torch.cuda.stream(stream):
            for _ in range(3):
                step()
            plan.check(stream)
            ms = 0.0
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
            plan.check(stream)
        row = {"value": steps * flop_step / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
               "us_per_step": ms * 1e3 / steps}
        if ref:
            errs = {}
            for i, n in enumerate(ns):
                M, e = ref[n]
                errs[str(n)] = oracle.rel_frobenius(outs[i].cpu().numpy().astype(np.float64),
                                                    int(lgs[i].item()), M, e)
            row["rel_frobenius_vs_f64"] = errs
            row["within_2e-5_ceil_log2_n"] = all(errs[str(n)] <= stated_tolerance(n) for n in ns)
        table[prec] = row
        plan.close()
    return {"workload": wk["desc"], "api": "one matpow_batched call over the 4 powers",
            "l2": "flushed between timed steps (256 MB write)", "paths": table}


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
    # the powers' results side by side in one allocation (one copy back per step)
    out_all = torch.empty((len(ns),) + tuple(A.shape), dtype=torch.float32, device=dev)
    outs = [out_all[i] for i in range(len(ns))]
    lgs = torch.zeros(len(ns), dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    plan = mpw.Plan(N, prec, device=local, tile_table=tile_table_path(args))
    plan.set_option(mpw.OPT_CHAIN, args.chain_mode)

    def step(s):
        if args.api == "batched" and len(ns) > 1:  # the powers side by side, one matpow_batched call
            st = mpw.matpow_batched(plan.h, [A] * len(ns), [N] * len(ns), ns, outs, lgs, s)
            if st != 0:
                mpw._check(st, plan.h)
            return
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
    errs = errors_of(wk, A_host, ns, outs, lgs) if rank == 0 and not args.no_check else {}
    # ---- the plain FP32 SIMT path on the same workload (the comparator of the
    # metric) and, for the large power, the plain BF16 path
    fp32 = bf16 = table2 = None
    if world == 1 and prec != "fp32" and not args.no_fp32:
        fp32 = path_compare(args, wk, A, A_host, flush, stream, value, "fp32")
        if N > 1024 and prec != "bf16":
            bf16 = path_compare(args, wk, A, A_host, flush, stream, value, "bf16")
    if world == 1 and N > 1024 and not args.no_config2:
        table2 = config2_table(args, dev, flush, stream)

    # ---- end to end through the C-ABI with host buffers
    A_pin = torch.from_numpy(A_host).pin_memory()
    out_pin = torch.empty(tuple(out_all.shape), dtype=torch.float32).pin_memory()
    lg_pin = torch.zeros(len(ns), dtype=torch.int64).pin_memory()
    e2e_steps = max(args.steps, 3)
    with torch.cuda.stream(stream):
        def e2e_step():
            A.copy_(A_pin, non_blocking=True)
            step(stream)
            out_pin.copy_(out_all, non_blocking=True)
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
    kind = mpw.KERNEL_SIMT if prec == "fp32" else mpw.KERNEL_TC
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
    products = PRODUCTS[prec]
    if kind == mpw.KERNEL_TC:
        achieved = kflop * products / (kms * 1e-3) / 1e12
        peak = peaks["bf16_tflops"]
        exact = prec in ("bf16x3", "bf16x6")
        chain_max = 768 if prec == "bf16x6" else 1024
        kname = (("tc_chain_split_kernel (split-K clusters) or tc_chain_kernel" if args.chain_mode == 1
                  else "tc_chain_kernel") if exact and 64 < N <= chain_max and args.chain_mode else
                 "tc_fxb_kernel" if exact else "tc_gemm_kernel")
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": kname, "peak_source": peak_src + " bf16 burst",
                "counted": "%d bfloat16 product(s) per term" % int(products)}
        if peaks.get("bf16_tflops_sustained"):
            roof["frac_of_sustained"] = achieved / peaks["bf16_tflops_sustained"]
    else:
        # float32 FFMA peak, measured by the library's register-only probe
        peak, psrc = fp32_peak(local)
        achieved = kflop / (kms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "simt_gemm" if kind == mpw.KERNEL_SIMT else "tiny_chain",
                "peak_source": psrc}
        if kind == mpw.KERNEL_TINY:
            # the chain is a dependent sequence of products on the SMs of one
            # CTA (N <= 32) or one four-CTA cluster: their share of the peak
            sms = 4 if N > 32 else 1
            roof["sms_used"] = sms
            roof["frac_of_sms_used"] = achieved / (peak * sms / 152)
    roof["launches_timed"] = kl
    roof["avg_launch_us"] = kms * 1e3 / max(kl, 1)
    tr = TRAFFIC.get((args.workload, prec))
    if tr:
        roof["traffic"] = tr[0]
        roof["traffic_source"] = tr[1]
    latency = None
    if N <= 64 and len(ns) == 1:
        # a latency-bound power: the distribution of one call's device time
        # (CUDA events around each call, 1000 calls back to back, L2 warm)
        reps = 1000
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(reps)]
        with torch.cuda.stream(stream):
            for a, b in pairs:
                a.record(stream)
                step(stream)
                b.record(stream)
            torch.cuda.synchronize()
        us = sorted(a.elapsed_time(b) * 1e3 for a, b in pairs)
        latency = {"unit": "us", "p50": us[reps // 2], "p99": us[int(reps * 0.99)], "min": us[0], "reps": reps,
                   "note": "per call, back to back, L2 warm"}

    if rank != 0:
        return
    cb = cpu_sample(wk, budget_s=args.cpu_budget, A=A_host) if world == 1 and not args.no_cpu else None
    line = {
        "metric": "matpow effective TFLOP/s", "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[prec],
        "data": "synthetic",
        "config": config_for(args, wk, world),
        "rel_frobenius_vs_f64": errs,
        "fp32_simt_same_workload": fp32,
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
    if bf16:
        line["bf16_same_workload"] = bf16
    if table2:
        line["n512_gaussian_all_paths"] = table2
    if latency:
        line["latency"] = latency
    print(json.dumps(line))
    plan.close()


def run_modp(args, wk, world, rank, local):
    """A^n mod p through matpow_mod_p (exact byte-sliced tensor-core products)."""
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    from paper_1204_3052_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_src = load_peaks()
    N, ns, pm = wk["N"], wk["ns"], wk["p"]
    flop_step = sum(gemm_count(n) for n in ns) * 2.0 * N ** 3
    A_host = wl.modp_uniform(N, pm, 0)
    A = torch.from_numpy(A_host.view(np.int32)).to(dev)
    outs = [torch.empty_like(A) for _ in ns]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    plan = mpw.Plan(N, "fp32", device=local)

    def step(s):
        for i, n in enumerate(ns):
            st = mpw.matpow_mod_p(plan.h, A, N, n, pm, outs[i], s)
            if st != 0:
                mpw._check(st, plan.h)

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
            flush.zero_()
            evs[k][0].record(stream)
            step(stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        barrier(world)
        clocks = sampler.stop()
        launches = plan.launch_count() - launches0
        st = plan.sync(stream)
    t_ms = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in evs), dev)
    value = world * args.steps * flop_step / (t_ms * 1e-3) / 1e12
    exact = None
    if rank == 0 and not args.no_check:
        import oracle
        exact = True
        for i, n in enumerate(ns):
            want, _ = oracle.matpow_modp(A_host, n, pm)
            got = outs[i].cpu().numpy().view(np.uint32).astype(np.uint64)
            exact = exact and bool(np.array_equal(got, want))
    # e2e: host input in, result out, through the C-ABI
    A_pin = torch.from_numpy(A_host.view(np.int32)).pin_memory()
    outs_pin = [torch.empty(A_host.shape, dtype=torch.int32).pin_memory() for _ in ns]
    e2e_steps = max(args.steps, 3)
    with torch.cuda.stream(stream):
        def e2e_step():
            A.copy_(A_pin, non_blocking=True)
            step(stream)
            for i in range(len(ns)):
                outs_pin[i].copy_(outs[i], non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(world, e0.elapsed_time(e1), dev)
    # dominant kernel: per-launch CUDA-event time of the mod-p products
    plan.set_option(mpw.OPT_TIMING, 1)
    with torch.cuda.stream(stream):
        plan.kernel_time(mpw.KERNEL_MODP, reset=True)
        for _ in range(max(args.steps, 3)):
            flush.zero_()
            step(stream)
        torch.cuda.synchronize()
        kl, kms, kflop = plan.kernel_time(mpw.KERNEL_MODP, reset=True)
    plan.set_option(mpw.OPT_TIMING, 0)
    plan.close()
    # four byte-slice products per product: 4 x 2N^3 bfloat16 tensor flop
    achieved = 4.0 * kflop / (kms * 1e-3) / 1e12
    roof = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
            "frac": achieved / peaks["bf16_tflops"], "traffic": None, "kernel": "tc_modp_kernel",
            "peak_source": peak_src + " bf16 burst", "counted": "4 bfloat16 byte-slice products per term",
            "launches_timed": kl, "avg_launch_us": kms * 1e3 / max(kl, 1)}
    tr = TRAFFIC.get((args.workload, args.precision))
    if tr:
        roof["traffic"], roof["traffic_source"] = tr
    if rank != 0:
        return
    cb = cpu_sample_modp(wk, args.cpu_budget) if world == 1 and not args.no_cpu else None
    line = {"metric": "matpow effective TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 mod p",
            "data": "synthetic", "config": config_for(args, wk, world),
            "bit_exact_vs_oracle": exact, "status": st, "wall_s_timed": wall, "clocks": clocks,
            "e2e": {"value": e2e_steps * flop_step / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": int(A_host.nbytes),
                    "d2h_bytes_per_step": int(A_host.nbytes * len(ns))},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cb}
    print(json.dumps(line))


def run_expm(args, wk, world, rank, local):
    """e^A through matpow_expm (scaling and squaring on the product and
    squaring kernels)."""
    import torch
    from paper_1204_3052_gb300 import matpow as mpw

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_src = load_peaks()
    N = wk["N"]
    A_host = expm_input(wk)
    flop_step = expm_flop(A_host)
    A = torch.from_numpy(A_host).to(dev)
    out = torch.empty_like(A)
    lg = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    plan = mpw.Plan(N, args.precision, device=local, tile_table=tile_table_path(args))

    def step(s):
        st = mpw.matpow_expm(plan.h, A, N, out, lg, s)
        if st != 0:
            mpw._check(st, plan.h)

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
            flush.zero_()
            evs[k][0].record(stream)
            step(stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        barrier(world)
        clocks = sampler.stop()
        launches = plan.launch_count() - launches0
        st = plan.sync(stream)
    t_ms = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in evs), dev)
    value = world * args.steps * flop_step / (t_ms * 1e-3) / 1e12
    errs = None
    if rank == 0 and not args.no_check:
        import oracle
        want = oracle.expm_f64(A_host)
        got = np.ldexp(out.cpu().numpy().astype(np.float64), int(lg.item()))
        s = oracle.expm_scaling(A_host, 1.0)
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        errs = {"rel_frobenius": err, "stated": 2e-5 * (s + 1), "within_2e-5_(s+1)": err <= 2e-5 * (s + 1)}
    # e2e: host input in, result (mantissa and exponent) out, through the C-ABI
    A_pin = torch.from_numpy(A_host).pin_memory()
    out_pin = torch.empty(A_host.shape, dtype=torch.float32).pin_memory()
    lg_pin = torch.zeros(1, dtype=torch.int64).pin_memory()
    e2e_steps = max(args.steps, 3)
    with torch.cuda.stream(stream):
        def e2e_step():
            A.copy_(A_pin, non_blocking=True)
            step(stream)
            out_pin.copy_(out, non_blocking=True)
            lg_pin.copy_(lg, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(world, e0.elapsed_time(e1), dev)
    # tensor-core kernels (products and squarings): per-launch CUDA-event time
    plan.set_option(mpw.OPT_TIMING, 1)
    kind = mpw.KERNEL_TC if args.precision != "fp32" else mpw.KERNEL_SIMT
    with torch.cuda.stream(stream):
        plan.kernel_time(kind, reset=True)
        for _ in range(max(args.steps, 3)):
            flush.zero_()
            step(stream)
        torch.cuda.synchronize()
        kl, kms, kflop = plan.kernel_time(kind, reset=True)
    plan.set_option(mpw.OPT_TIMING, 0)
    plan.close()
    products = PRODUCTS[args.precision]
    if kind == mpw.KERNEL_TC:
        achieved = kflop * products / (kms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                "frac": achieved / peaks["bf16_tflops"], "traffic": None,
                "kernel": "tc_chain kernels and tc_fxb_kernel (powers, products, squarings)",
                "peak_source": peak_src + " bf16 burst", "counted": "%d bfloat16 product(s) per term" % products}
    else:
        peak, psrc = fp32_peak(local)
        achieved = kflop / (kms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "simt_gemm", "peak_source": psrc}
    roof["launches_timed"] = kl
    roof["avg_launch_us"] = kms * 1e3 / max(kl, 1)
    roof["kernel_share_of_step"] = kms / max(args.steps, 3) / (t_ms / args.steps)
    if rank != 0:
        return
    cb = cpu_sample_expm(wk, args.cpu_budget) if world == 1 and not args.no_cpu else None
    line = {"metric": "matpow effective TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic", "config": config_for(args, wk, world),
            "rel_frobenius_vs_f64": errs, "status": st, "wall_s_timed": wall, "clocks": clocks,
            "e2e": {"value": e2e_steps * flop_step / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": int(A_host.nbytes), "d2h_bytes_per_step": int(A_host.nbytes) + 8},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cb}
    print(json.dumps(line))


def run_naive(args, wk, world, rank, local):
    """Square-and-multiply vs the naive GPU method (n - 1 products R <- R A, one
    launch each; the paper's Sec. 4.2 method) with the same product kernels,
    at the paper's orders and powers; the paper reports ~44x on a C2050."""
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    from paper_1204_3052_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    fast = mpw.Plan(max(wk["Ns"]), args.precision, device=local)
    naive = mpw.Plan(max(wk["Ns"]), args.precision, device=local)
    naive.set_option(mpw.OPT_NAIVE, 1)
    naive.set_option(mpw.OPT_TINY_MAX, 0)
    rows, t_fast, t_naive, flop_alg = [], 0.0, 0.0, 0.0
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    for N in wk["Ns"]:
        A = torch.from_numpy(wl.gaussian(N, 0)).to(dev)
        out = torch.empty_like(A)
        lg = torch.zeros(1, dtype=torch.int64, device=dev)
        for n in wk["ns_list"]:
            ms = {}
            for name, plan, reps in (("fast", fast, max(args.steps, 3)), ("naive", naive, 2)):
                with torch.cuda.stream(stream):
                    for _ in range(args.warmup if name == "fast" else 1):
                        mpw._check(mpw.matpow_f32(plan.h, A, N, n, out, lg, stream), plan.h)
                    plan.check(stream)
                    tot = 0.0
                    for _ in range(reps):
                        flush.zero_()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        mpw._check(mpw.matpow_f32(plan.h, A, N, n, out, lg, stream), plan.h)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        tot += e0.elapsed_time(e1)
                    plan.check(stream)
                ms[name] = tot / reps
            t_fast += ms["fast"]
            t_naive += ms["naive"]
            flop_alg += gemm_count(n) * 2.0 * N ** 3
            rows.append({"N": N, "n": n, "square_multiply_ms": ms["fast"], "naive_ms": ms["naive"],
                         "speedup": ms["naive"] / ms["fast"], "products": [gemm_count(n), n - 1]})
    clocks = sampler.stop()
    fast.close()
    naive.close()
    if rank != 0:
        return
    value = flop_alg / (t_fast * 1e-3) / 1e12
    line = {"metric": "matpow effective TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_fast,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic", "config": config_for(args, wk, world),
            "vs_naive_gpu": rows, "speedup_over_naive_total": t_naive / t_fast,
            "paper_context": "Sec. 5.2 reports about 44x over its naive GPU kernel on a Tesla C2050",
            "clocks": clocks,
            "e2e": None, "gpu_launches": None, "roofline": None, "cpu_baseline": None}
    print(json.dumps(line))


def batch_roofline_ms(Ns, ns, prec, peaks) -> float:
    """Lower bound of a batch step's level launches: level L holds the L-th
    level of every matrix's schedule (its squaring and, if that bit of n is
    set, R <- R P), and takes at least max(algorithmic bytes / HBM copy
    bandwidth, tensor flop / bf16 peak); the bound is the sum over levels.
    Algorithmic bytes of a product: read each distinct operand's slice planes
    once (2 B per slice per element), write the next ones; orders N <= 64
    (the on-chip small-order chain) are left out."""
    planes = {"bf16x6": 3, "bf16x3": 2, "bf16": 1, "fp32": 2}[prec]
    per_prod = PRODUCTS[prec]
    levels = {}
    for N, n in zip(Ns, ns):
        if N <= 64 or n < 2:
            continue
        bits, L, have_r = n, 0, False
        while bits:
            ops = []
            if bits & 1:
                if have_r:
                    ops.append(False)  # R <- R P (distinct operands)
                have_r = True
            bits >>= 1
            if bits:
                ops.append(True)  # P <- P P
            if ops:
                by, fl = levels.get(L, (0.0, 0.0))
                for sq in ops:
                    by += 2.0 * planes * N * N * ((1 if sq else 2) + 1)
                    fl += per_prod * 2.0 * N ** 3
                levels[L] = (by, fl)
                L += 1
    bw = peaks.get("hbm_gbs", 6704.5) * 1e9
    tf = peaks["bf16_tflops"] * 1e12
    return sum(max(by / bw, fl / tf) for by, fl in levels.values()) * 1e3


def run_batched(args, wk, world, rank, local):
    """Config 3: one matpow_batched call over an uneven batch per step."""
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    from paper_1204_3052_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_src = load_peaks()
    bd = wl.batched_draw(count=wk["count"], seed=0, n_max=wk["n_max"])
    Ns = [int(x) for x in bd.Ns]
    ns = [int(x) for x in bd.ns]
    hostA = [wl.gaussian(N, int(sd)) for N, sd in zip(Ns, bd.seeds)]
    # the batch packed into one allocation per direction, as a caller that
    # stages it with one copy would hold it; the API takes one pointer per matrix
    offs = np.cumsum([0] + [N * N for N in Ns])
    dbuf = torch.empty(int(offs[-1]), dtype=torch.float32, device=dev)
    obuf = torch.empty_like(dbuf)
    dA = [dbuf[int(o):int(o) + N * N].view(N, N) for o, N in zip(offs[:-1], Ns)]
    outs = [obuf[int(o):int(o) + N * N].view(N, N) for o, N in zip(offs[:-1], Ns)]
    hbuf = np.concatenate([a.reshape(-1) for a in hostA])
    dbuf.copy_(torch.from_numpy(hbuf))
    lg = torch.zeros(len(dA), dtype=torch.int64, device=dev)
    flop_step = sum(gemm_count(n) * 2.0 * N ** 3 for N, n in zip(Ns, ns))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    plan = mpw.Plan(max(Ns), args.precision, device=local, tile_table=tile_table_path(args))

    def step(s):
        mpw._check(mpw.matpow_batched(plan.h, dA, Ns, ns, outs, lg, s), plan.h)

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
        l0 = plan.launch_count()
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            step(stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        barrier(world)
        clocks = sampler.stop()
        launches = plan.launch_count() - l0
        st = plan.sync(stream)
    t_ms = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in evs), dev)
    value = world * args.steps * flop_step / (t_ms * 1e-3) / 1e12
    # accuracy on a sample of the batch
    errs = {}
    if rank == 0 and not args.no_check:
        import oracle
        for i in range(0, len(Ns), max(1, len(Ns) // 16)):
            M, e, _ = oracle.matpow_f64(hostA[i], ns[i])
            errs["N%d_n%d" % (Ns[i], ns[i])] = oracle.rel_frobenius(
                outs[i].cpu().numpy(), int(lg[i].item()), M, e)
    # end to end: inputs from pinned host memory, results back, inside the timed region
    pinA = torch.from_numpy(hbuf).pin_memory()
    pinO = torch.empty(obuf.shape, dtype=torch.float32).pin_memory()
    pinL = torch.zeros(len(dA), dtype=torch.int64).pin_memory()
    with torch.cuda.stream(stream):
        def e2e_step():
            dbuf.copy_(pinA, non_blocking=True)
            step(stream)
            pinO.copy_(obuf, non_blocking=True)
            pinL.copy_(lg, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(max(args.steps, 2)):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / max(args.steps, 2)
    ref_out = pinO.clone()
    # the same end to end with the batch in K contiguous chunks of equal work,
    # one plan each (a plan's workspace and captured launch graph belong to
    # one call): chunk k's input copy (one copy stream) and chunk k - 1's
    # result copy (another) overlap the products of the chunks around them;
    # the products run in order on the step's stream
    K = 4
    work = np.cumsum([gemm_count(n) * float(N) ** 3 for N, n in zip(Ns, ns)])
    cuts = sorted({int(np.searchsorted(work, work[-1] * (k + 1) / K)) + 1 for k in range(K - 1)})
    bounds = [0] + [c for c in cuts if 0 < c < len(Ns)] + [len(Ns)]
    chunks = [(b0, b1) for b0, b1 in zip(bounds[:-1], bounds[1:]) if b1 > b0]
    cplans = [mpw.Plan(max(Ns[b0:b1]), args.precision, device=local, tile_table=tile_table_path(args))
              for b0, b1 in chunks]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def e2e_pipelined():
        go = torch.cuda.Event()
        go.record(stream)
        s_in.wait_event(go)
        ready = []
        for b0, b1 in chunks:
            o0, o1 = int(offs[b0]), int(offs[b1])
            with torch.cuda.stream(s_in):
                dbuf[o0:o1].copy_(pinA[o0:o1], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s_in)
            ready.append(ev)
        for (b0, b1), ev, cp in zip(chunks, ready, cplans):
            o0, o1 = int(offs[b0]), int(offs[b1])
            stream.wait_event(ev)
            mpw._check(mpw.matpow_batched(cp.h, dA[b0:b1], Ns[b0:b1], ns[b0:b1], outs[b0:b1], lg[b0:b1],
                                          stream), cp.h)
            done = torch.cuda.Event()
            done.record(stream)
            s_out.wait_event(done)
            with torch.cuda.stream(s_out):
                pinO[o0:o1].copy_(obuf[o0:o1], non_blocking=True)
                pinL[b0:b1].copy_(lg[b0:b1], non_blocking=True)
        fin = torch.cuda.Event()
        fin.record(s_out)
        stream.wait_event(fin)

    with torch.cuda.stream(stream):
        e2e_pipelined()
        torch.cuda.synchronize()
        pipe_equal = bool(torch.equal(pinO, ref_out))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(max(args.steps, 2)):
            e2e_pipelined()
        e1.record(stream)
        torch.cuda.synchronize()
        pipe_ms = e0.elapsed_time(e1) / max(args.steps, 2)
    for cp in cplans:
        cp.check(stream)
        cp.close()
    # dominant kernel timing
    plan.set_option(mpw.OPT_TIMING, 1)
    kind = mpw.KERNEL_TC if args.precision != "fp32" else mpw.KERNEL_SIMT
    with torch.cuda.stream(stream):
        plan.kernel_time(kind, reset=True)
        for _ in range(2):
            flush.zero_()
            step(stream)
        torch.cuda.synchronize()
        kl, kms, kflop = plan.kernel_time(kind, reset=True)
        tl, tms, tflop = plan.kernel_time(mpw.KERNEL_TINY, reset=True)
    plan.set_option(mpw.OPT_TIMING, 0)
    products = PRODUCTS[args.precision]
    achieved = kflop * products / (kms * 1e-3) / 1e12 if kms else 0.0
    roof = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
            "frac": achieved / peaks["bf16_tflops"], "traffic": None,
            "kernel": "tc_fxb_persist_kernel (persistent grouped level launches, N > 64)",
            "peak_source": peak_src + " bf16 burst", "launches_timed": kl,
            "avg_launch_us": kms * 1e3 / max(kl, 1),
            "tiny_chain_share_ms": tms / 2, "level_kernels_ms": kms / 2}
    tr = TRAFFIC.get((args.workload, args.precision))
    if tr:
        roof["traffic"], roof["traffic_source"] = tr
    roof["level_roofline_bound_ms"] = batch_roofline_ms(Ns, ns, args.precision, peaks)
    if rank != 0:
        return
    cb = None
    if world == 1 and not args.no_cpu:
        import oracle
        cores = oracle.set_threads(0)
        t0 = time.perf_counter()
        done, i = 0.0, 0
        while time.perf_counter() - t0 < args.cpu_budget and i < len(Ns):
            oracle.matpow_f64(hostA[i], ns[i])
            done += gemm_count(ns[i]) * 2.0 * Ns[i] ** 3
            i += 1
        dt = time.perf_counter() - t0
        cb = {"value": done / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
              "sample": "float64 square-and-multiply of the first %d matrices of the batch (%.1f s)" % (i, dt)}
    line = {"metric": "matpow effective TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": config_for(args, wk, world),
            "rel_frobenius_vs_f64": errs, "status": st, "wall_s_timed": wall, "clocks": clocks,
            "e2e": {"value": flop_step / (min(e2e_ms, pipe_ms) * 1e-3) / 1e12, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": int(sum(a.nbytes for a in hostA)),
                    "d2h_bytes_per_step": int(sum(a.nbytes for a in hostA) + 8 * len(Ns)),
                    "method": ("%d chunks of equal work, copies overlapped on two copy streams"
                               % len(chunks)) if pipe_ms < e2e_ms else "one call, copies before and after",
                    "ms_per_step": min(e2e_ms, pipe_ms),
                    "one_call": {"value": flop_step / (e2e_ms * 1e-3) / 1e12, "ms_per_step": e2e_ms},
                    "chunked": {"value": flop_step / (pipe_ms * 1e-3) / 1e12, "ms_per_step": pipe_ms,
                                "chunks": len(chunks), "results_equal_one_call": pipe_equal}},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cb}
    print(json.dumps(line))
    plan.close()


def _lindley(arrivals, service):
    """Latencies of a single FIFO server (one request at a time) by Lindley's
    recursion: start_i = max(arrival_i, finish_(i-1)), latency = finish - arrival."""
    lat = np.empty(len(arrivals))
    free = 0.0
    for i, (t, d) in enumerate(zip(arrivals, service)):
        start = max(t, free)
        free = start + d
        lat[i] = free - t
    return lat


def run_serving(args, wk, world, rank, local):
    """Config 5 (scaled): requests through matpow_submit / matpow_poll.

    1. capacity: the whole stream submitted at once (closed burst), req/s;
    2. Poisson arrivals at 0.5, 0.8, 1.0 and 1.2 x that capacity on the first
       `sweep_count` requests: served req/s, p50 and p99 latency;
    3. comparator: the same requests one at a time through single-request
       plan calls (each timed with CUDA events), and the p50/p99 an unbatched
       FIFO server with those service times would give at the same loads.
    """
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    from paper_1204_3052_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    count = wk["count"]
    sweep_count = min(count, args.sweep_count) if args.sweep_count > 0 else count
    base_rate = 1000.0
    reqs = wl.serving_stream(count=count, seed=0, rate_per_s=base_rate)
    # inputs drawn on a thread pool and moved to the device as they come; the
    # host keeps only the matrices the oracle checks (every mod-p request with
    # N <= 256, and float requests with N <= 512, n <= 1024, one in 50)
    check_mod = [r.kind == 1 and r.N <= 256 for r in reqs]
    check_flt = [r.kind == 0 and r.N <= 512 and r.n <= 1024 for r in reqs]
    kf = [i for i, c in enumerate(check_flt) if c][::50]
    check_flt = [False] * count
    for i in kf:
        check_flt[i] = True
    host = [None] * count
    dA, outs, lgs = [], [], []
    from concurrent.futures import ThreadPoolExecutor
    t_gen = time.perf_counter()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        for i, a in enumerate(ex.map(wl.request_matrix, reqs)):
            r = reqs[i]
            t = torch.from_numpy(a.view(np.int32) if r.kind else a).to(dev)
            dA.append(t)
            outs.append(torch.empty_like(t))
            lgs.append(torch.zeros(1, dtype=torch.int64, device=dev) if r.kind == 0 else None)
            if check_mod[i] or check_flt[i]:
                host[i] = a
    t_gen = time.perf_counter() - t_gen
    flop = sum(gemm_count(r.n) * 2.0 * r.N ** 3 for r in reqs)
    server = mpw.Server(2048, args.precision, device=local, hbm_budget_bytes=16 << 30,
                        max_inflight=256, max_queue=count + 16)

    def submit(i):
        r = reqs[i]
        return server.submit(dA[i], r.n, outs[i], kind=r.kind, p=r.p, log2_scale=lgs[i])

    def drain(tickets):
        bad = 0
        for t in tickets:
            if server.wait(t, timeout_s=600) != mpw.OK:
                bad += 1
        torch.cuda.synchronize()
        return bad

    # warm-up requests (not timed)
    drain([submit(i) for i in range(min(8, count))])
    # ---- 1. capacity: closed burst of the whole stream
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    n0 = len(server.latencies_us())
    t0 = time.perf_counter()
    bad = drain([submit(i) for i in range(count)])
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    capacity = count / wall
    burst_lat = np.asarray(server.latencies_us()[n0:])
    # ---- 2. Poisson load sweep
    sweep = []
    arr0 = np.array([r.t_arrival for r in reqs[:sweep_count]])
    for f in args.sweep:
        rate = f * capacity
        arr = arr0 * base_rate / rate
        n0 = len(server.latencies_us())
        t0 = time.perf_counter()
        tickets = []
        for i in range(sweep_count):
            delay = arr[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(submit(i))
        bad += drain(tickets)
        w = time.perf_counter() - t0
        lat = np.asarray(server.latencies_us()[n0:])
        sweep.append({"load": f, "offered_req_per_s": rate, "served_req_per_s": sweep_count / w,
                      "p50_ms": float(np.percentile(lat, 50) / 1e3),
                      "p99_ms": float(np.percentile(lat, 99) / 1e3)})
    server.close()
    # exact mod-p requests checked against the oracle (those with N <= 256),
    # and a sample of float requests (their errors reported)
    checked = mism = 0
    ferrs = []
    if not args.no_check:
        import oracle
        for i, (r, a, o) in enumerate(zip(reqs, host, outs)):
            if check_mod[i]:
                want, _ = oracle.matpow_modp(a, r.n, r.p)
                checked += 1
                mism += int(not np.array_equal(o.cpu().numpy().view(np.uint32).astype(np.uint64), want))
            elif check_flt[i]:
                M, e, _ = oracle.matpow_f64(a, r.n)
                err = oracle.rel_frobenius(o.cpu().numpy(), int(lgs[i].item()), M, e)
                ferrs.append((err, err <= stated_tolerance(r.n)))
    # ---- 3. unbatched comparator: single-request calls, one at a time
    plan_f = mpw.Plan(2048, args.precision, device=local)
    plan_m = mpw.Plan(2048, "fp32", device=local)
    stream = torch.cuda.current_stream(dev)

    def single(i):
        r = reqs[i]
        if r.kind:
            mpw._check(mpw.matpow_mod_p(plan_m.h, dA[i], r.N, r.n, r.p, outs[i]), plan_m.h)
        else:
            mpw._check(mpw.matpow_f32(plan_f.h, dA[i], r.N, r.n, outs[i], lgs[i]), plan_f.h)

    for i in range(min(8, sweep_count)):
        single(i)
    torch.cuda.synchronize()
    svc = np.empty(sweep_count)
    for i in range(sweep_count):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        single(i)
        e1.record(stream)
        e1.synchronize()
        svc[i] = e0.elapsed_time(e1) * 1e-3
    plan_f.close()
    plan_m.close()
    unb_cap = sweep_count / svc.sum()
    unb = {"req_per_s": unb_cap, "ms_per_request_mean": float(svc.mean() * 1e3),
           "note": "device time of each request alone through matpow_f32 / matpow_mod_p; "
                   "latencies of a one-at-a-time FIFO server with these service times"}
    unb["sweep"] = []
    for f in args.sweep:
        rate = f * capacity
        lat = _lindley(arr0 * base_rate / rate, svc)
        unb["sweep"].append({"load": f, "offered_req_per_s": rate,
                             "p50_ms": float(np.percentile(lat, 50) * 1e3),
                             "p99_ms": float(np.percentile(lat, 99) * 1e3)})
    if rank != 0:
        return
    line = {"metric": "matpow serving req/s", "value": capacity, "unit": "req/s", "n_gpus": world,
            "steps": 1, "warmup": 8, "ms_per_step": wall * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": config_for(args, wk, world),
            "p50_ms": float(np.percentile(burst_lat, 50) / 1e3) if burst_lat.size else None,
            "p99_ms": float(np.percentile(burst_lat, 99) / 1e3) if burst_lat.size else None,
            "latency_note": "p50/p99 of the closed burst (queueing included); see load_sweep",
            "load_sweep": sweep, "effective_tflops": flop / wall / 1e12, "failed_requests": bad,
            "modp_checked": checked, "modp_mismatches": mism,
            "float_checked": len(ferrs),
            "float_max_rel_frobenius": max((e for e, _ in ferrs), default=None),
            "float_within_2e-5_ceil_log2_n": sum(ok for _, ok in ferrs),
            "input_generation_s": t_gen,
            "unbatched": unb, "speedup_over_unbatched": capacity / unb_cap,
            "clocks": clocks,
            "e2e": {"value": capacity, "unit": "req/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0,
                    "note": "inputs resident; submit-to-completion through the public API"},
            "gpu_launches": None, "roofline": None, "cpu_baseline": None}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large8192")
    ap.add_argument("--precision", choices=sorted(DTYPE), default=None,
                    help="default: the cheapest path that meets the stated error on the workload "
                         "(bf16x6 for Gaussian inputs, bf16x3 for stochastic ones)")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 SIMT (and plain BF16) comparators")
    ap.add_argument("--no-config2", action="store_true",
                    help="large workloads: skip the N=512 table of every float path")
    ap.add_argument("--api", choices=["batched", "single"], default="batched",
                    help="single-matrix workloads: all powers in one matpow_batched call (default) or "
                         "one matpow_f32 call per power")
    ap.add_argument("--chain-mode", type=int, choices=[0, 1, 2], default=1,
                    help="whole-chain kernel for N <= 1024: 1 with split-K (default), 2 without, "
                         "0 level-by-level launches")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--ref-budget", type=float, default=5.0)
    ap.add_argument("--sweep", type=float, nargs="*", default=[0.5, 0.8, 1.0, 1.2],
                    help="serving: offered loads as fractions of the measured capacity")
    ap.add_argument("--sweep-count", type=int, default=0,
                    help="serving: requests per load point (0: the whole stream)")
    ap.add_argument("--tile-table", default="default",
                    help="'default' (the tuned table shipped with the package, if present), 'none' "
                         "(built-in rules) or a tile-table JSON file")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wk = WORKLOADS[args.workload]
    if args.precision is None:
        args.precision = wk["prec"]
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, wk, world, rank)
    elif wk.get("kind") == "batched":
        run_batched(args, wk, world, rank, local)
    elif wk.get("kind") == "serving":
        run_serving(args, wk, world, rank, local)
    elif wk.get("kind") == "modp":
        run_modp(args, wk, world, rank, local)
    elif wk.get("kind") == "expm":
        run_expm(args, wk, world, rank, local)
    elif wk.get("kind") == "naive":
        run_naive(args, wk, world, rank, local)
    else:
        run_ours(args, wk, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
