"""Seeded synthetic inputs for the integer matrix power A^n.

This module is shared by the CUDA path's callers (tests, bench, smoke) and by
the CPU oracle's callers.  It holds none of the method's arithmetic: it only
draws matrices, exponents and request streams.  Every draw comes from numpy's
Philox-4x32-10 counter-based generator (Salmon et al., SC'11) keyed by the
seed, and Gaussian entries are made by the Box-Muller transform in float64 from
Philox uniforms, so the bits do not depend on numpy's normal sampler.

The paper tests "dense" matrices of orders 64..512 and powers 64..1024
(Sec. 5.2, Tables 1-3) without naming a value distribution; the recipes below
stand in for them:

* ``gaussian(N)``: entries N(0, 1/N) rounded to float32 (spectral radius ~1).
* ``stochastic_exact(N)``: row-stochastic from U[0,1) draws, made exact in
  float32 (each row sums to exactly 1, so the largest eigenvalue is exactly 1
  and "row sums of A^n stay 1" holds for the true power, not only approximately).
* ``modp_uniform(N, p)``: integer entries U{0..p-1}.
* ``batched_draw``: the uneven batch (N in {16,...,256}, n log-uniform in [1,4096]).
* ``serving_stream``: Poisson arrivals, N log-uniform in [8,2048], n
  log-uniform in [1,2^30], 90% float / 10% mod p.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

P_DEFAULT = 65521  # largest prime below 2^16


def rng(seed: int) -> np.random.Generator:
    """Philox-4x32-10 stream keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(int(seed)))


def _box_muller(g: np.random.Generator, count: int) -> np.ndarray:
    """``count`` standard normals (float64) from Philox uniforms."""
    m = (count + 1) // 2
    u1 = 1.0 - g.random(m)  # (0, 1]
    u2 = g.random(m)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
    return z[:count]


def gaussian(N: int, seed: int = 0) -> np.ndarray:
    """N x N float32 matrix with entries N(0, 1/N), row-major."""
    g = rng(seed)
    z = _box_muller(g, N * N) / math.sqrt(max(N, 1))
    return z.astype(np.float32).reshape(N, N)


def stochastic_exact(N: int, seed: int = 0) -> np.ndarray:
    """N x N float32 row-stochastic matrix whose rows sum to exactly 1.

    Row i draws u_ij ~ U[0,1), turns them into integer weights q_ij that sum to
    2^s_i exactly (rounding residual added to the row's largest weight) and
    stores a_ij = q_ij * 2^-s_i.  s_i is chosen so that every q_ij < 2^24, so
    each a_ij is exact in float32 and the exact row sum is 1.
    """
    g = rng(seed)
    u = g.random((N, N))
    out = np.empty((N, N), dtype=np.float32)
    for i in range(N):
        row = u[i]
        tot = row.sum()
        if tot <= 0.0:
            row = np.ones(N)
            tot = float(N)
        share = row / tot
        smax = share.max()
        s = int(math.floor(math.log2((2.0 ** 23) / smax)))
        q = np.rint(share * 2.0 ** s).astype(np.int64)
        resid = (1 << s) - int(q.sum())
        q[int(np.argmax(q))] += resid
        assert q.min() >= 0 and q.max() < (1 << 24)
        out[i] = (q.astype(np.float64) * 2.0 ** (-s)).astype(np.float32)
    return out


def uniform01(N: int, seed: int = 0) -> np.ndarray:
    """N x N float32 matrix with entries U[0,1)."""
    return rng(seed).random((N, N)).astype(np.float32)


def modp_uniform(N: int, p: int = P_DEFAULT, seed: int = 0) -> np.ndarray:
    """N x N uint32 matrix with entries U{0..p-1}."""
    return rng(seed).integers(0, p, size=(N, N), dtype=np.uint64).astype(np.uint32)


def log_uniform_int(g: np.random.Generator, lo: int, hi: int, size: int) -> np.ndarray:
    """floor(lo * ((hi+1)/lo)^U) clipped to [lo, hi], U ~ U[0,1)."""
    u = g.random(size)
    v = np.floor(lo * np.exp(u * math.log((hi + 1) / lo))).astype(np.int64)
    return np.clip(v, lo, hi)


@dataclass
class BatchDraw:
    Ns: np.ndarray      # int64, matrix orders
    ns: np.ndarray      # uint64, exponents
    seeds: np.ndarray   # per-matrix seeds for the entries


def batched_draw(count: int = 4096, seed: int = 0, n_max: int = 4096,
                 N_step: int = 16, N_classes: int = 16) -> BatchDraw:
    """Uneven batch: N = N_step * U{1..N_classes}, n log-uniform in [1, n_max]."""
    g = rng(seed)
    Ns = N_step * g.integers(1, N_classes + 1, size=count)
    ns = log_uniform_int(g, 1, n_max, count).astype(np.uint64)
    seeds = g.integers(0, 2 ** 62, size=count)
    return BatchDraw(Ns.astype(np.int64), ns, seeds.astype(np.int64))


@dataclass
class Request:
    t_arrival: float    # seconds from stream start
    N: int
    n: int
    kind: int           # 0 = float32 A^n, 1 = A^n mod p
    p: int
    seed: int


def serving_stream(count: int = 20000, seed: int = 0, rate_per_s: float = 1000.0,
                   N_lo: int = 8, N_hi: int = 2048, n_hi: int = 2 ** 30,
                   frac_modp: float = 0.10, p: int = P_DEFAULT) -> list[Request]:
    """Poisson request stream (exponential inter-arrivals at ``rate_per_s``)."""
    g = rng(seed)
    gaps = -np.log(1.0 - g.random(count)) / rate_per_s
    t = np.cumsum(gaps)
    Ns = log_uniform_int(g, N_lo, N_hi, count)
    ns = log_uniform_int(g, 1, n_hi, count)
    kinds = (g.random(count) < frac_modp).astype(np.int64)
    seeds = g.integers(0, 2 ** 62, size=count)
    return [Request(float(t[i]), int(Ns[i]), int(ns[i]), int(kinds[i]), p, int(seeds[i]))
            for i in range(count)]


def request_matrix(req: Request) -> np.ndarray:
    """Entries of a serving request: N(0,1/N) float32, or U{0..p-1} uint32."""
    if req.kind == 0:
        return gaussian(req.N, req.seed)
    return modp_uniform(req.N, req.p, req.seed)


# ---- structured matrices with known powers (test inputs) -------------------

def fibonacci_blocks(N: int) -> np.ndarray:
    """Block-diagonal copies of [[1,1],[1,0]] (a trailing 1x1 block is [1])."""
    A = np.zeros((N, N), dtype=np.float32)
    for b in range(0, N - 1, 2):
        A[b, b] = A[b, b + 1] = A[b + 1, b] = 1.0
    if N % 2:
        A[N - 1, N - 1] = 1.0
    return A


def rotation(theta: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s], [s, c]], dtype=np.float64)


def shift(N: int) -> np.ndarray:
    """Nilpotent upper shift: ones on the first superdiagonal."""
    return np.eye(N, k=1, dtype=np.float32)


def permutation(N: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Random permutation matrix P (P[i, perm[i]] = 1) and its index vector."""
    perm = rng(seed).permutation(N)
    P = np.zeros((N, N), dtype=np.float32)
    P[np.arange(N), perm] = 1.0
    return P, perm
