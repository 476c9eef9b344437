"""Python binding of libmatpow (include/matpow.h).

Argument marshalling only: every function here forwards to the C-ABI entry
point of the same name in ``libmatpow.so``, which runs all of the work in its
own CUDA kernels.  PyTorch supplies device memory and streams.  There is no
CPU fallback: if the library cannot be loaded (or built with nvcc) every call
raises.

Thin same-name wrappers (``matpow_plan``, ``matpow_f32``, ``matpow_mod_p``,
``matpow_batched``, ``matpow_sync``, ``matpow_submit``, ``matpow_poll``, ...)
take torch tensors or raw integers; the ``Plan`` and ``Server`` classes add
ownership and convenience on top of them.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmatpow.so")

OK, EINVAL, ENOMEM, ECUDA, EAGAIN, EBUSY, ETIMEDOUT, ERANGE, EUNSUPPORTED = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EAGAIN", "EBUSY", "ETIMEDOUT", "ERANGE",
                "EUNSUPPORTED"]
FP32_SIMT, BF16, BF16X3, BF16X6 = 0, 1, 2, 3
PRECISIONS = {"fp32": FP32_SIMT, "fp32_simt": FP32_SIMT, "bf16": BF16, "bf16x3": BF16X3,
              "bf16x6": BF16X6}
OPT_GRAPHS, OPT_TIMING, OPT_TINY_MAX, OPT_TILE, OPT_SPLIT, OPT_CHAIN, OPT_MODP_TC, OPT_PERSIST, OPT_NAIVE = (
    1, 2, 3, 4, 5, 6, 7, 8, 9)
OPT_PAIR = 10
KERNEL_SIMT, KERNEL_TC, KERNEL_TINY, KERNEL_MODP, KERNEL_AUX = range(5)

EXPORTS = [
    "matpow_plan", "matpow_workspace_size", "matpow_plan_destroy", "matpow_last_error",
    "matpow_plan_set_option", "matpow_f32", "matpow_mod_p", "matpow_batched", "matpow_sync",
    "matpow_gemm_count", "matpow_kernel_time", "matpow_launch_count", "matpow_server_create",
    "matpow_submit", "matpow_poll", "matpow_server_latencies", "matpow_server_destroy",
    "matpow_f32_noalloc", "matpow_selftest_wait_timeout", "matpow_expm",
    "matpow_plan_set_tile_table", "matpow_plan_load_tile_table", "matpow_tile_table_parse",
    "matpow_tile_rule_lookup", "matpow_selftest_ffma", "matpow_plan_sm_count", "matpow_host_accessible",
]

# The tile table tuned on a GB300 (written by autotune.py); plans load it when
# asked (Plan(tile_table=DEFAULT_TILE_TABLE)).
DEFAULT_TILE_TABLE = os.path.join(_HERE, "tile_table_gb300.json")
TILE_FIELDS = ("n_lo", "n_hi", "precision", "bn", "split_k", "chain", "persist")


class MatpowError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, msg))
        self.status = status


class ServerDesc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_n", ctypes.c_int), ("precision", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("max_queue", ctypes.c_int)]


class TileRule(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in TILE_FIELDS]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f in TILE_FIELDS}


class Request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n", ctypes.c_uint64), ("kind", ctypes.c_int),
                ("p", ctypes.c_uint32), ("dA", ctypes.c_void_p), ("dOut", ctypes.c_void_p),
                ("dLog2Scale", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmatpow.so (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise OSError("libmatpow.so is not built: run __graft_entry__.build()")
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32, u64, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t)
        protos = {
            "matpow_plan": (i32, [ctypes.POINTER(vp), i32, i32, sz, i32]),
            "matpow_workspace_size": (sz, [i32, i32]),
            "matpow_plan_destroy": (i32, [vp]),
            "matpow_last_error": (ctypes.c_char_p, [vp]),
            "matpow_plan_set_option": (i32, [vp, i32, i64]),
            "matpow_f32": (i32, [vp, vp, i32, u64, vp, vp, vp]),
            "matpow_mod_p": (i32, [vp, vp, i32, u64, u32, vp, vp]),
            "matpow_batched": (i32, [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(i32),
                                     ctypes.POINTER(u64), ctypes.POINTER(vp), vp, vp]),
            "matpow_sync": (i32, [vp, vp]),
            "matpow_gemm_count": (i32, [u64]),
            "matpow_kernel_time": (i32, [vp, i32, ctypes.POINTER(i64),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), i32]),
            "matpow_launch_count": (i64, [vp]),
            "matpow_server_create": (i32, [ctypes.POINTER(vp), ctypes.POINTER(ServerDesc)]),
            "matpow_submit": (i32, [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]),
            "matpow_poll": (i32, [vp, u64, u32]),
            "matpow_server_latencies": (i64, [vp, ctypes.POINTER(ctypes.c_double), i64]),
            "matpow_server_destroy": (i32, [vp]),
            "matpow_f32_noalloc": (i32, [vp, i32, u64, vp, vp, vp]),
            "matpow_selftest_wait_timeout": (i32, [vp, u64, vp]),
            "matpow_expm": (i32, [vp, vp, i32, vp, vp, vp]),
            "matpow_selftest_ffma": (i32, [vp, i64, vp]),
            "matpow_plan_sm_count": (i32, [vp]),
            "matpow_host_accessible": (i32, [vp, i32]),
            "matpow_plan_set_tile_table": (i32, [vp, ctypes.POINTER(TileRule), i32]),
            "matpow_plan_load_tile_table": (i32, [vp, ctypes.c_char_p]),
            "matpow_tile_table_parse": (i32, [ctypes.c_char_p, ctypes.POINTER(TileRule), i32,
                                              ctypes.POINTER(i32)]),
            "matpow_tile_rule_lookup": (i32, [ctypes.POINTER(TileRule), i32, i32, i32,
                                              ctypes.POINTER(TileRule)]),
        }
        for name, (res, args) in protos.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(x) -> int:
    """Device address of a torch tensor (or an int address)."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st: int, plan=None):
    if st != OK:
        lib = load()
        msg = lib.matpow_last_error(plan)
        raise MatpowError(st, msg.decode() if msg else "")


# ---- same-name wrappers ---------------------------------------------------------

def matpow_plan(max_n: int, precision=FP32_SIMT, workspace_bytes: int = 0, device: int = 0) -> int:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = ctypes.c_void_p()
    _check(load().matpow_plan(ctypes.byref(h), int(max_n), int(precision), int(workspace_bytes),
                              int(device)))
    return h.value


def matpow_workspace_size(max_n: int, precision=FP32_SIMT) -> int:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return int(load().matpow_workspace_size(int(max_n), int(precision)))


def matpow_plan_destroy(plan: int) -> None:
    _check(load().matpow_plan_destroy(plan))


def matpow_plan_set_option(plan: int, key: int, value: int) -> None:
    _check(load().matpow_plan_set_option(plan, int(key), int(value)), plan)


def matpow_f32(plan: int, A, N: int, n: int, out, log2_scale=None, stream=None) -> int:
    return load().matpow_f32(plan, _ptr(A), int(N), int(n), _ptr(out), _ptr(log2_scale),
                             _stream(stream))


def matpow_f32_noalloc(A, N: int, n: int, out, log2_scale=None, stream=None) -> int:
    return load().matpow_f32_noalloc(_ptr(A), int(N), int(n), _ptr(out), _ptr(log2_scale),
                                     _stream(stream))


def matpow_mod_p(plan: int, A, N: int, n: int, p: int, out, stream=None) -> int:
    return load().matpow_mod_p(plan, _ptr(A), int(N), int(n), int(p), _ptr(out), _stream(stream))


def matpow_batched(plan: int, As: Sequence, Ns: Sequence[int], ns: Sequence[int], outs: Sequence,
                   log2_scale=None, stream=None) -> int:
    c = len(As)
    a = (ctypes.c_void_p * c)(*[_ptr(x) for x in As])
    o = (ctypes.c_void_p * c)(*[_ptr(x) for x in outs])
    Nn = (ctypes.c_int * c)(*[int(x) for x in Ns])
    nn = (ctypes.c_uint64 * c)(*[int(x) for x in ns])
    return load().matpow_batched(plan, c, a, Nn, nn, o, _ptr(log2_scale), _stream(stream))


def matpow_sync(plan: int, stream=None) -> int:
    return load().matpow_sync(plan, _stream(stream))


def matpow_expm(plan: int, A, N: int, out, log2_scale=None, stream=None) -> int:
    return load().matpow_expm(plan, _ptr(A), N, _ptr(out), _ptr(log2_scale), _stream(stream))


def matpow_selftest_wait_timeout(plan: int, budget_ns: int, stream=None) -> int:
    return load().matpow_selftest_wait_timeout(plan, int(budget_ns), _stream(stream))


def _rules_array(rules):
    arr = (TileRule * max(len(rules), 1))()
    for i, r in enumerate(rules):
        d = dict(r)
        if isinstance(d.get("precision"), str):
            d["precision"] = PRECISIONS[d["precision"]]
        for f in TILE_FIELDS:
            setattr(arr[i], f, int(d.get(f, -1)))
    return arr


def matpow_plan_set_tile_table(plan: int, rules) -> int:
    """rules: a list of dicts with the fields of matpow_tile_rule (precision may be a name)."""
    return load().matpow_plan_set_tile_table(plan, _rules_array(rules), len(rules))


def matpow_plan_load_tile_table(plan: int, path: str) -> int:
    return load().matpow_plan_load_tile_table(plan, os.fsencode(path))


def matpow_tile_table_parse(text: str):
    """(status, [rule dicts]) of tile-table JSON text, parsed by the library."""
    lib = load()
    n = ctypes.c_int()
    st = lib.matpow_tile_table_parse(text.encode(), None, 0, ctypes.byref(n))
    if st != OK:
        return st, []
    arr = (TileRule * max(n.value, 1))()
    st = lib.matpow_tile_table_parse(text.encode(), arr, n.value, ctypes.byref(n))
    return st, [arr[i].as_dict() for i in range(n.value)]


def matpow_tile_rule_lookup(rules, precision, N: int):
    """(status, rule dict) the library selects from `rules` for (precision, N)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    out = TileRule()
    st = load().matpow_tile_rule_lookup(_rules_array(rules), len(rules), int(precision), int(N),
                                        ctypes.byref(out))
    return st, out.as_dict()


def matpow_selftest_ffma(plan: int, iters: int, stream=None) -> int:
    return load().matpow_selftest_ffma(plan, int(iters), _stream(stream))


def matpow_plan_sm_count(plan: int) -> int:
    return int(load().matpow_plan_sm_count(plan))


def matpow_host_accessible(buf, device: int = 0) -> bool:
    """Whether `device` addresses `buf` (a tensor or an address) at the same
    pointer, so that it may stand where a call takes a device matrix."""
    return bool(load().matpow_host_accessible(_ptr(buf), int(device)))


def measure_fp32_peak(plan: int, iters: int = 1 << 16, reps: int = 5, stream=None) -> float:
    """FP32 FFMA TFLOP/s of the plan's device: the best of `reps` timed runs
    of matpow_selftest_ffma (CUDA events on the stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    flop = 2.0 * 8 * iters * 256 * 8 * matpow_plan_sm_count(plan)
    best = 0.0
    _check(matpow_selftest_ffma(plan, iters, s), plan)  # warm-up
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check(matpow_selftest_ffma(plan, iters, s), plan)
        e1.record(s)
        e1.synchronize()
        best = max(best, flop / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def matpow_gemm_count(n: int) -> int:
    return int(load().matpow_gemm_count(int(n)))


def matpow_kernel_time(plan: int, kind: int, reset: bool = False):
    launches = ctypes.c_int64()
    ms = ctypes.c_double()
    flop = ctypes.c_double()
    _check(load().matpow_kernel_time(plan, int(kind), ctypes.byref(launches), ctypes.byref(ms),
                                     ctypes.byref(flop), int(reset)), plan)
    return int(launches.value), float(ms.value), float(flop.value)


def matpow_launch_count(plan: int) -> int:
    return int(load().matpow_launch_count(plan))


def matpow_server_create(device: int = 0, max_n: int = 2048, precision=BF16X3,
                         hbm_budget_bytes: int = 8 << 30, max_inflight: int = 256,
                         max_queue: int = 1 << 16) -> int:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    d = ServerDesc(device, max_n, precision, hbm_budget_bytes, max_inflight, max_queue)
    h = ctypes.c_void_p()
    _check(load().matpow_server_create(ctypes.byref(h), ctypes.byref(d)))
    return h.value


def matpow_submit(server: int, N: int, n: int, kind: int, p: int, A, out, log2_scale=None):
    r = Request(int(N), int(n), int(kind), int(p), _ptr(A), _ptr(out), _ptr(log2_scale))
    t = ctypes.c_uint64()
    st = load().matpow_submit(server, ctypes.byref(r), ctypes.byref(t))
    return st, int(t.value)


def matpow_poll(server: int, ticket: int, timeout_us: int = 0) -> int:
    return load().matpow_poll(server, int(ticket), int(timeout_us))


def matpow_server_latencies(server: int, cap: int) -> np.ndarray:
    buf = np.zeros(max(int(cap), 1), dtype=np.float64)
    k = load().matpow_server_latencies(server, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       int(cap))
    return buf[:k]


def matpow_server_destroy(server: int) -> None:
    _check(load().matpow_server_destroy(server))


# ---- convenience classes ----------------------------------------------------------

class Plan:
    """Owns one libmatpow plan; tensors are torch CUDA tensors."""

    def __init__(self, max_n: int, precision="fp32", device: int = 0, workspace_bytes: int = 0,
                 tile_table: Optional[str] = None):
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.device = device
        self.max_n = max_n
        self.h = matpow_plan(max_n, self.precision, workspace_bytes, device)
        if tile_table:
            self.load_tile_table(tile_table)

    def load_tile_table(self, path: str):
        """Launch shapes per order range from a tile-table JSON file."""
        _check(matpow_plan_load_tile_table(self.h, path), self.h)

    def set_tile_table(self, rules):
        _check(matpow_plan_set_tile_table(self.h, rules), self.h)

    def close(self):
        if self.h:
            matpow_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: int, value: int):
        matpow_plan_set_option(self.h, key, value)

    def f32(self, A, n: int, out=None, mantissa: bool = False, stream=None):
        """A^n (float32).  Returns out, or (out, log2 tensor) with mantissa=True."""
        import torch
        N = A.shape[0]
        if out is None:
            out = torch.empty_like(A)
        lg = torch.zeros(1, dtype=torch.int64, device=A.device) if mantissa else None
        _check(matpow_f32(self.h, A, N, n, out, lg, stream), self.h)
        return (out, lg) if mantissa else out

    def expm(self, A, out=None, mantissa: bool = False, stream=None):
        """e^A (float32).  Returns out, or (out, log2 tensor) with mantissa=True."""
        import torch
        N = A.shape[0]
        if out is None:
            out = torch.empty_like(A)
        lg = torch.zeros(1, dtype=torch.int64, device=A.device) if mantissa else None
        _check(matpow_expm(self.h, A, N, out, lg, stream), self.h)
        return (out, lg) if mantissa else out

    def mod_p(self, A, n: int, p: int, out=None, stream=None):
        import torch
        N = A.shape[0]
        if out is None:
            out = torch.empty_like(A)
        _check(matpow_mod_p(self.h, A, N, n, p, out, stream), self.h)
        return out

    def batched(self, As, ns, outs=None, log2=None, stream=None):
        import torch
        if outs is None:
            outs = [torch.empty_like(a) for a in As]
        _check(matpow_batched(self.h, As, [a.shape[0] for a in As], ns, outs, log2, stream), self.h)
        return outs

    def sync(self, stream=None) -> int:
        return matpow_sync(self.h, stream)

    def check(self, stream=None):
        _check(self.sync(stream), self.h)

    def kernel_time(self, kind: int, reset: bool = False):
        return matpow_kernel_time(self.h, kind, reset)

    def launch_count(self) -> int:
        return matpow_launch_count(self.h)


class Server:
    """Owns one libmatpow request server (continuous batching)."""

    def __init__(self, max_n: int, precision="fp32", device: int = 0,
                 hbm_budget_bytes: int = 1 << 30, max_inflight: int = 64, max_queue: int = 1 << 16):
        self.h = matpow_server_create(device, max_n, precision, hbm_budget_bytes, max_inflight,
                                      max_queue)

    def submit(self, A, n: int, out, kind: int = 0, p: int = 0, log2_scale=None) -> int:
        """Queue A^n (kind 0, float32) or A^n mod p (kind 1, uint32); returns the ticket."""
        st, t = matpow_submit(self.h, A.shape[0], n, kind, p, A, out, log2_scale)
        if st != OK:
            _check(st)
        return t

    def poll(self, ticket: int, timeout_us: int = 0) -> int:
        return matpow_poll(self.h, ticket, timeout_us)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        import time
        t_end = time.time() + timeout_s
        while True:
            st = self.poll(ticket, 100000)
            if st not in (EAGAIN, ETIMEDOUT) or time.time() > t_end:
                return st

    def latencies_us(self, cap: int = 1 << 20):
        return matpow_server_latencies(self.h, cap)

    def close(self):
        if self.h:
            matpow_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
