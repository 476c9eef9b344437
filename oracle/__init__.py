"""CPU oracle for the integer matrix power A^n (arXiv 1204.3052).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this package.  It shares no code with the CUDA library and imports nothing
from it; the two meet only through the seeded inputs of
``paper_1204_3052_gb300.workloads``, which the callers pass in.

Functions and the passage each follows:

* ``gemm_f64``, ``gemm_modp``: the plain triple-loop product (Sec. 4.1), in C;
  ``gemm_rows_f64`` the same loop over a range of rows (a timing sample).
* ``matpow_f64(A, n, mode)``: A^n in float64, as mantissa and power-of-two
  exponent.  ``mode="sqmul"`` is the log2(n)-product method (Sec. 4.3),
  ``mode="brute"`` the n-1 repeated products (Sec. 4.1, 4.2).
* ``matpow_modp(A, n, p, mode)``: the same over the integers mod p, exact.
* ``schedule(n)``: the right-to-left binary level plan and the product count
  G(n) = floor(log2 n) + popcount(n) - 1 (Sec. 4.3's "log(N)" products).
* ``rel_frobenius``: the error measure ||X - Y||_F / ||Y||_F in float64.
* ``stationary(A)``: the limit 1 pi^T of A^n for a positive row-stochastic A,
  by float64 power iteration (a closed form for large n).
* ``fp32_sqmul(A, n)``: the same square-and-multiply with every product
  rounded to float32 (numpy float32 matmul as the product step).  An error
  yardstick, not a parity target; pinned by exact integer chains, a diagonal
  chain against the scalar float32 chain, and a product whose float32 sum
  rounds differently from the float64 one.
* ``perturbed_sqmul(A, n, rel, seed)``: the float64 chain with a seeded
  normwise perturbation of size rel added to every stored partial product:
  the sensitivity of A^n's chain to storage errors of that size (the
  float32-class floor of the tests' float bounds where 2e-5 ceil(log2 n) is
  out of reach).  Pinned by a scalar closed form, linearity in rel and
  rel = 0 giving the oracle's power.
* ``round_bf16``, ``split_bf16``: round-to-nearest-even to bfloat16 (8
  significant bits) and the two-part split x ~ hi + lo, hi = bf16(x),
  lo = bf16(x - hi).
* ``fixed_slices(X, block)``: the fixed-point split of a matrix scaled by
  the power-of-two maximum 2^s of each block x block tile (block=None: one
  scale for the whole matrix): u = X 2^(8-s), a1 = rint(u),
  a2 = rint(256 (u - a1)), so X ~ 2^(s-16) (256 a1 + a2) with integer slices
  |a1| <= 256, |a2| <= 128.  ``fixed_slices_n(X, block, k)`` continues the
  same recurrence to k slices (a_(j+1) = rint(256 * remainder)), so
  X ~ 2^(s-8k) sum_j 256^(k-1-j) a_j.
* ``expm_f64(A)``: the matrix exponential e^A in float64 from the series
  definition by scaling and squaring (Moler and Van Loan 2003, method 3):
  e^A = (sum_k B^k / k!)^(2^s), B = A / 2^s, ||B||_1 <= 1/2, 18 terms.
  ``expm_fp32_ps(A)``: the float32 yardstick of the GPU evaluation (degree-11
  Taylor polynomial in Paterson-Stockmeyer form, float32 products), and
  ``expm_emu_ps(A, precision)`` the same with emulated tensor-core operand
  rounding; parity unpinned.
* ``emu_sqmul(A, n, precision)``: the square-and-multiply chain with the
  operand rounding of a tensor-core precision emulated on the CPU ("bf16":
  one bfloat16 product; "bf16x3": hi*hi + hi*lo + lo*hi of floating
  bfloat16 parts; "bf16x3fx": a1*b1 + a1*b2 + a2*b1 of the fixed-point
  slices with one scale per matrix; "bf16x3blk": the same with one scale per
  64 x 64 block; "bf16x6blk": three block-scaled slices and the six products
  a_i b_j with i + j <= 2; products and sums in float64, each result rounded
  to float32).  An error yardstick for the lower-precision paths, not a
  parity target.  Pinned (tests/test_oracle_yardsticks.py) by products on
  the precisions' exact grids (equal to the exact product), products with
  one operand off the grid (equal to the exact product of the operand
  rounded to the grid by a one-step formula), exact integer chains, and a
  diagonal chain against the scalar chain; a dropped slice product, a wrong
  slice weight, a skipped rounding, a transposed operand or a dropped
  multiply step each fail one of them.

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``): Fibonacci, rotation,
diagonal, nilpotent shift, permutation and identity closed forms; A^(m+k) =
A^m A^k; exact row sums of stochastic powers and their 1 pi^T limit; brute
force against square-and-multiply; the mod-p path against Python integers.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "matpow_oracle.c")
_LIB = os.path.join(_HERE, "libmatpow_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (IEEE float64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            up = ctypes.POINTER(ctypes.c_uint64)
            ip = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_gemm_f64.argtypes = [ctypes.c_int, dp, dp, dp]
            lib.oracle_gemm_f64.restype = None
            lib.oracle_matpow_f64.argtypes = [ctypes.c_int, dp, ctypes.c_uint64, ctypes.c_int,
                                              dp, ip, ip]
            lib.oracle_matpow_f64.restype = ctypes.c_int
            lib.oracle_gemm_rows_f64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            lib.oracle_gemm_rows_f64.restype = None
            lib.oracle_gemm_modp.argtypes = [ctypes.c_int, up, up, ctypes.c_uint64, up]
            lib.oracle_gemm_modp.restype = None
            lib.oracle_matpow_modp.argtypes = [ctypes.c_int, up, ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_int, up, ip]
            lib.oracle_matpow_modp.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(threads: int) -> int:
    """OpenMP threads for the product loops (<= 0: all cores); returns the count."""
    return _load().oracle_set_threads(int(threads))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _uptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _square(A) -> int:
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    return A.shape[0]


def gemm_f64(A, B) -> np.ndarray:
    """A @ B by the plain triple loop (Sec. 4.1), float64."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    N = _square(A)
    C = np.empty((N, N), dtype=np.float64)
    _load().oracle_gemm_f64(N, _dptr(A), _dptr(B), _dptr(C))
    return C


def gemm_rows_f64(A, B, r0: int, r1: int) -> np.ndarray:
    """Rows r0 .. r1-1 of A @ B by the same triple loop as ``gemm_f64`` (each
    entry equal to the full product's); a bounded sample of a large product."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    N = _square(A)
    if not 0 <= r0 <= r1 <= N:
        raise ValueError("row range outside the matrix")
    C = np.empty((r1 - r0, N), dtype=np.float64)
    _load().oracle_gemm_rows_f64(N, int(r0), int(r1), _dptr(A), _dptr(B), _dptr(C))
    return C


def gemm_modp(A, B, p: int) -> np.ndarray:
    """(A @ B) mod p by the plain triple loop, exact."""
    A = np.ascontiguousarray(A, dtype=np.uint64)
    B = np.ascontiguousarray(B, dtype=np.uint64)
    N = _square(A)
    C = np.empty((N, N), dtype=np.uint64)
    _load().oracle_gemm_modp(N, _uptr(A), _uptr(B), int(p), _uptr(C))
    return C


_MODES = {"sqmul": 0, "brute": 1}


def matpow_f64(A, n: int, mode: str = "sqmul"):
    """A^n as (M, e, gemms): A^n = M * 2**e with max|M| in [0.5, 1) or M = 0."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    N = _square(A)
    M = np.empty((N, N), dtype=np.float64)
    e = ctypes.c_int64(0)
    g = ctypes.c_int64(0)
    rc = _load().oracle_matpow_f64(N, _dptr(A), int(n), _MODES[mode], _dptr(M),
                                   ctypes.byref(e), ctypes.byref(g))
    if rc != 0:
        raise RuntimeError("oracle_matpow_f64 failed: %d" % rc)
    return M, int(e.value), int(g.value)


def matpow_value(A, n: int, mode: str = "sqmul") -> np.ndarray:
    """A^n in float64 (M * 2**e; may overflow to inf for huge results)."""
    M, e, _ = matpow_f64(A, n, mode)
    return np.ldexp(M, e)


def matpow_modp(A, n: int, p: int, mode: str = "sqmul"):
    """(A^n mod p, gemms) with entries of A in [0, p)."""
    A = np.ascontiguousarray(A, dtype=np.uint64)
    N = _square(A)
    out = np.empty((N, N), dtype=np.uint64)
    g = ctypes.c_int64(0)
    rc = _load().oracle_matpow_modp(N, _uptr(A), int(n), int(p), _MODES[mode], _uptr(out),
                                    ctypes.byref(g))
    if rc != 0:
        raise RuntimeError("oracle_matpow_modp failed: %d" % rc)
    return out, int(g.value)


def schedule(n: int):
    """Right-to-left binary plan for A^n (Sec. 4.3).

    Returns a list of levels; level k is a tuple (multiply, square) of
    booleans: ``multiply`` when bit k of n is set and a partial result already
    exists (R <- R * P), ``square`` when a higher bit remains (P <- P * P).
    The first set bit only copies P into R.
    """
    levels = []
    have_r = False
    bits = int(n)
    while bits:
        mul = False
        if bits & 1:
            if have_r:
                mul = True
            have_r = True
        bits >>= 1
        levels.append((mul, bits != 0))
    return levels


def gemm_count(n: int) -> int:
    """G(n): products the square-and-multiply method performs for A^n."""
    return sum(int(m) + int(s) for m, s in schedule(n))


def rel_frobenius(M, e, M_ref, e_ref) -> float:
    """||M*2^e - M_ref*2^e_ref||_F / ||M_ref*2^e_ref||_F, in float64.

    Both sides are brought to the reference's exponent first, so results far
    outside the float range compare without overflow.
    """
    X = np.ldexp(np.asarray(M, dtype=np.float64), int(e) - int(e_ref))
    Y = np.asarray(M_ref, dtype=np.float64)
    den = np.linalg.norm(Y)
    num = np.linalg.norm(X - Y)
    if den == 0.0:
        return 0.0 if num == 0.0 else math.inf
    return float(num / den)


def stationary(A, iters: int = 200000, tol: float = 1e-15) -> np.ndarray:
    """pi with pi^T A = pi^T, sum(pi) = 1, by float64 power iteration.

    For a positive row-stochastic A, A^n -> 1 pi^T as n grows; the rate is
    |lambda_2|^n.
    """
    A = np.asarray(A, dtype=np.float64)
    N = _square(A)
    pi = np.full(N, 1.0 / N)
    for _ in range(iters):
        nxt = pi @ A
        nxt /= nxt.sum()
        if np.max(np.abs(nxt - pi)) <= tol:
            return nxt
        pi = nxt
    return pi


def _normalise32(X, e):
    """(X 2^-s, e + s) with s the frexp exponent of max|X| (exact power of two)."""
    mx = float(np.max(np.abs(X))) if X.size else 0.0
    if mx == 0.0 or not math.isfinite(mx):
        return X, e
    _, s = math.frexp(mx)
    return np.ldexp(X, -s).astype(np.float32), e + s


def _sqmul_chain(A, n: int, product):
    """Square-and-multiply (Sec. 4.3) over the level plan ``schedule(n)``
    with ``product(X, Y)`` (float32 result) as the product step and an exact
    power-of-two rescale after every product.  Returns (M, e): A^n ~ M 2^e."""
    A = np.asarray(A, dtype=np.float32)
    N = _square(A)
    if n == 0:
        return np.eye(N, dtype=np.float32), 0
    P, ep = _normalise32(A.copy(), 0)
    R, er = None, 0
    for k, (mul, sq) in enumerate(schedule(n)):
        if mul:
            R, er = _normalise32(product(R, P), er + ep)
        elif R is None and (int(n) >> k) & 1:  # the first set bit copies P
            R, er = P.copy(), ep
        if sq:
            P, ep = _normalise32(product(P, P), 2 * ep)
    return R, er


def _fp32_product(X, Y):
    """float32 product (numpy float32 matmul): the product step of fp32_sqmul."""
    return np.matmul(np.asarray(X, dtype=np.float32), np.asarray(Y, dtype=np.float32))


def fp32_sqmul(A, n: int):
    """Square-and-multiply with float32 products (error yardstick; parity unpinned).

    Returns (M, e): A^n ~ M * 2**e, each product rounded to float32 by numpy's
    float32 matmul and rescaled by an exact power of two.
    """
    return _sqmul_chain(A, n, lambda X, Y: _fp32_product(X, Y))


def perturbed_sqmul(A, n: int, rel: float, seed: int):
    """The float64 square-and-multiply chain (Sec. 4.3; numpy float64 matmul
    as the product step) with every stored partial product disturbed
    normwise: after the exact power-of-two rescale that puts max|X| in
    [0.5, 1), each entry gets rel * r added, r uniform in [-1, 1) drawn from
    numpy's default generator seeded with ``seed`` (one draw per entry, in
    row-major order, stored product after stored product).  The result's
    deviation from ``matpow_f64`` measures how far relative errors of size
    rel in each stored matrix carry through the chain (its first-order
    sensitivity), whatever arithmetic produced those errors; rel = 2^-24 is
    the storage precision of a float32-class result.  Returns (M, e):
    A^n ~ M 2^e."""
    g = np.random.default_rng(seed)
    A = np.asarray(A, dtype=np.float64)
    N = _square(A)

    def store(X, e):
        mx = float(np.max(np.abs(X))) if X.size else 0.0
        if mx == 0.0 or not math.isfinite(mx):
            return X, e
        _, s = math.frexp(mx)
        X = np.ldexp(X, -s)
        return X + rel * g.uniform(-1.0, 1.0, X.shape), e + s

    if n == 0:
        return np.eye(N), 0
    P, ep = store(A.copy(), 0)
    R, er = None, 0
    for k, (mul, sq) in enumerate(schedule(n)):
        if mul:
            R, er = store(R @ P, er + ep)
        elif R is None and (int(n) >> k) & 1:
            R, er = P.copy(), ep
        if sq:
            P, ep = store(P @ P, 2 * ep)
    return R, er


def round_bf16(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32.

    bfloat16 keeps the top 16 bits of a float32: add 0x7FFF plus the lowest
    kept bit to the 32-bit pattern and clear the low 16 bits.  Inputs are
    finite.
    """
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def split_bf16(x):
    """(hi, lo) with hi = bf16(x), lo = bf16(x - hi); x - hi is exact in float32."""
    x = np.asarray(x, dtype=np.float32)
    hi = round_bf16(x)
    lo = round_bf16((x - hi).astype(np.float32))
    return hi, lo


_rint = np.rint  # round half to even: the slices' rounding step


def fixed_slices(X, block=None):
    """(a1, a2, s): X ~ 2^(s-16) (256 a1 + a2), s the frexp exponent of max|X|
    over the whole matrix (block=None) or over each block x block tile (s is
    then an array of X's shape holding each entry's tile exponent)."""
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    if block is None:
        mx = float(np.max(np.abs(X))) if X.size else 0.0
        s = math.frexp(mx)[1] if mx > 0.0 else 0
    else:
        s = np.zeros(X.shape, dtype=np.int64)
        for i in range(0, X.shape[0], block):
            for j in range(0, X.shape[1], block):
                mx = float(np.max(np.abs(X[i:i + block, j:j + block])))
                s[i:i + block, j:j + block] = math.frexp(mx)[1] if mx > 0.0 else 0
    u = np.ldexp(X, 8 - s)
    a1 = _rint(u)
    a2 = _rint((u - a1) * 256.0)
    return a1, a2, s


def fixed_slices_n(X, block, k: int):
    """([a_0, ..., a_(k-1)], s): the k-slice fixed-point split of X with one
    frexp exponent per block x block tile (s has X's shape):
    u = X 2^(8-s), a_0 = rint(u), a_(j+1) = rint(256 (u_j - a_j)) with
    u_(j+1) = 256 (u_j - a_j); X ~ 2^(s-8k) sum_j 256^(k-1-j) a_j."""
    a1, _, s = fixed_slices(X, block)
    u = np.ldexp(np.asarray(X, dtype=np.float32).astype(np.float64), 8 - s)
    out = []
    for _ in range(k):
        a = _rint(u)
        out.append(a)
        u = (u - a) * 256.0
    return out, s


# Block fixed-point precisions: (slices per operand, the slice products
# a_i b_j kept).  Slice j of a matrix with block exponent s weighs 2^(s - 8 (j+1)).
SLICE_TERMS = {
    "bf16x3blk": (2, ((0, 0), (0, 1), (1, 0))),
    "bf16x6blk": (3, ((0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (2, 0))),
}
SLICE_BITS = 8


def _slice_weight_exp(s, j):
    """Exponent of slice j's weight for block exponent s: s - 8 (j + 1)."""
    return s - SLICE_BITS * (j + 1)


def _emu_product(X, Y, precision: str) -> np.ndarray:
    if precision in SLICE_TERMS:
        k, terms = SLICE_TERMS[precision]
        a, sx = fixed_slices_n(X, 64, k)
        b, sy = fixed_slices_n(Y, 64, k)
        x = [np.ldexp(a[j], _slice_weight_exp(sx, j)) for j in range(k)]
        y = [np.ldexp(b[j], _slice_weight_exp(sy, j)) for j in range(k)]
        P = np.zeros((x[0].shape[0], y[0].shape[1]))
        for i, j in terms:
            P += x[i] @ y[j]
        return P.astype(np.float32)
    if precision == "bf16x3fx":
        a1, a2, sx = fixed_slices(X)
        b1, b2, sy = fixed_slices(Y)
        T = a1 @ b1 + (a1 @ b2 + a2 @ b1) / 256.0
        return np.ldexp(T, sx + sy - 16).astype(np.float32)
    if precision == "bf16":
        P = round_bf16(X).astype(np.float64) @ round_bf16(Y).astype(np.float64)
    elif precision == "bf16x3":
        xh, xl = split_bf16(X)
        yh, yl = split_bf16(Y)
        xh, xl, yh, yl = (a.astype(np.float64) for a in (xh, xl, yh, yl))
        P = xh @ yh + xh @ yl + xl @ yh
    else:
        raise ValueError(precision)
    return P.astype(np.float32)


def emu_sqmul(A, n: int, precision: str):
    """Square-and-multiply with emulated tensor-core operand rounding (yardstick).

    Returns (M, e): A^n ~ M * 2**e.  The stored matrices keep float32 values,
    as the products' accumulators do; each product re-rounds its operands.
    """
    return _sqmul_chain(A, n, lambda X, Y: _emu_product(X, Y, precision))


# ---------------------------------------------------------------------------
# The matrix exponential e^A (the "scaling and squaring" use of the same
# squaring chain; Moler and Van Loan, "Nineteen dubious ways to compute the
# exponential of a matrix, twenty-five years later", SIAM Review 45 (2003),
# method 3).  Not part of arXiv 1204.3052, which means A^n by "matrix
# exponentiation"; this is the other common meaning, built on the same core.

def expm_scaling(A, theta: float):
    """s = max(0, ceil(log2(||A||_1 / theta))): the number of squarings that
    brings ||A / 2^s||_1 to at most theta (1-norm: the largest column sum)."""
    A = np.asarray(A, dtype=np.float64)
    nrm = float(np.max(np.sum(np.abs(A), axis=0))) if A.size else 0.0
    if not math.isfinite(nrm):
        raise ValueError("non-finite input")
    if nrm <= theta:
        return 0
    return max(0, math.ceil(math.log2(nrm / theta)))


def expm_f64(A, terms: int = 18):
    """e^A in float64 from its definition, the exponential series
    e^B = sum_k B^k / k!, applied to B = A / 2^s with ||B||_1 <= 1/2 (the
    terms past B^18 / 18! are below 2^-53 relative), then
    e^A = (e^B)^(2^s) by s squarings.  The series is summed by Horner's rule,
    T <- I + B T / k for k = terms .. 1; every product is the plain triple
    loop (gemm_f64)."""
    A = np.asarray(A, dtype=np.float64)
    N = _square(A)
    s = expm_scaling(A, 0.5)
    B = np.ldexp(A, -s)
    I = np.eye(N)
    T = I.copy()
    for k in range(terms, 0, -1):
        T = I + gemm_f64(B, T) / k
    for _ in range(s):
        T = gemm_f64(T, T)
    return T


def expm_emu_ps(A, precision: str):
    """``expm_fp32_ps`` with every product's operands rounded as a tensor-core
    precision would round them (``_emu_product``; the squarings by
    ``emu_sqmul``): the error yardstick of the lower-precision paths on the
    same evaluation (parity unpinned).  Returns (M, e)."""
    return expm_fp32_ps(A, lambda X, Y: _emu_product(X, Y, precision),
                        lambda T, n: emu_sqmul(T, n, precision))


def expm_fp32_ps(A, mul=None, power=None):
    """The float32-class yardstick of the GPU method (parity unpinned): s
    squarings for ||A / 2^s||_1 <= 1, the degree-11 Taylor polynomial of
    B = A / 2^s in Paterson-Stockmeyer form
        T = P0 + B^4 (P1 + B^4 P2),  Pj = sum_{i<4} B^i / (4j + i)!,
    with B^2, B^3, B^4 and the two outer products rounded to float32 (numpy
    float32 matmul) and the sums formed in float64 then rounded to float32,
    and T^(2^s) by float32 squarings.  Returns (M, e): e^A ~ M 2^e."""
    mul = mul or np.matmul
    power = power or fp32_sqmul
    A = np.asarray(A, dtype=np.float64)
    N = _square(A)
    s = expm_scaling(A, 1.0)
    B = np.ldexp(A, -s).astype(np.float32)
    B2 = mul(B, B)
    B3 = mul(B2, B)
    B4 = mul(B2, B2)
    I = np.eye(N)
    P = []
    for j in range(3):
        c = [1.0 / math.factorial(4 * j + i) for i in range(4)]
        P.append((c[0] * I + c[1] * B.astype(np.float64) + c[2] * B2.astype(np.float64)
                  + c[3] * B3.astype(np.float64)).astype(np.float32))
    Q = mul(B4, P[2])
    P1 = (P[1].astype(np.float64) + Q).astype(np.float32)
    R = mul(B4, P1)
    T = (P[0].astype(np.float64) + R).astype(np.float32)
    return power(T, 1 << s) if s > 0 else (T, 0)
