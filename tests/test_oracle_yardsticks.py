"""Pins for the oracle's error yardsticks (CPU only).

The yardsticks size the float tests' bounds: ``fp32_sqmul`` (float32
products), ``emu_sqmul`` (the tensor-core precisions' operand rounding
emulated) and ``perturbed_sqmul`` (the float64 chain with a normwise
perturbation of every stored product).  Each is fixed here against something
outside itself:

* products on a precision's exact grid equal the exact product (float64 sums
  that are exact by construction, rounded once to float32);
* products with one operand off the grid equal the exact product of that
  operand rounded to the grid by a one-step formula,
  rint(x 2^(b-s)) 2^(s-b) with s the block's frexp exponent and b its bits;
* exact integer chains equal the definition of A^n (Python-exact values);
* a diagonal chain equals the scalar square-and-multiply chain with the same
  rounding per product;
* the perturbation model's scalar case equals its closed form, and its
  deviation is linear in the perturbation size.

The second half plants one mistake at a time into the yardsticks (through the
tables and hooks they read: the kept slice products, the slice weights, the
rounding step, the float32 product, the level plan) and checks that one of
the pins above fails for each.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1204_3052_gb300 import workloads as wl


# ------------------------------------------------------------------ inputs

def _block_exponents(X, block=64):
    """frexp exponent of each block x block tile's maximum, broadcast to X's shape."""
    s = np.zeros(X.shape, dtype=np.int64)
    for i in range(0, X.shape[0], block):
        for j in range(0, X.shape[1], block):
            m = float(np.max(np.abs(X[i:i + block, j:j + block])))
            s[i:i + block, j:j + block] = math.frexp(m)[1] if m > 0 else 0
    return s


def _to_grid(X, bits, step=np.rint):
    """X rounded to each 64 x 64 block's 2^(s - bits) grid in one step (s from
    X itself).  step=np.trunc keeps every block inside its binade, so the
    result is on its own blocks' grid: the way grid inputs are built."""
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    s = _block_exponents(X)
    return np.ldexp(step(np.ldexp(X, bits - s)), s - bits)


def _on_grid(X, bits):
    return _to_grid(X, bits, np.trunc).astype(np.float32)


def _mat(seed, N=100, spread=4):
    """Nonsymmetric float32 matrix whose 64 x 64 blocks differ in scale by up
    to 2^spread: every product of two such matrices on grids of <= 24 bits has
    exact float64 sums (24 + 24 + spread + log2 N < 53 bits)."""
    g = wl.rng(seed)
    X = g.standard_normal((N, N))
    for i in range(0, N, 64):
        for j in range(0, N, 64):
            X[i:i + 64, j:j + 64] *= 2.0 ** int(g.integers(0, spread + 1))
    return X.astype(np.float32)


def _exact32(X, Y):
    return (np.asarray(X, np.float64) @ np.asarray(Y, np.float64)).astype(np.float32)


# ------------------------------------------------------------------ pin checks (return a list of failures)

def pins_block_products(prec):
    """Exactness and one-step rounding of the block fixed-point products."""
    bad = []
    prod = lambda X, Y: oracle._emu_product(X, Y, prec)
    top = 16 if prec == "bf16x3blk" else 24
    X, Y, Z = _mat(31), _mat(32), _mat(33)
    x8, y8 = _on_grid(X, 8), _on_grid(Y, 8)
    xt, yt = _on_grid(X, top), _on_grid(Y, top)
    # one operand with a single nonzero slice: every kept term i + 0 / 0 + j
    if not np.array_equal(prod(xt, y8), _exact32(xt, y8)):
        bad.append("top grid x 8-bit grid")
    if not np.array_equal(prod(x8, yt), _exact32(x8, yt)):
        bad.append("8-bit grid x top grid")
    # one operand off the grid: the product of its one-step rounding
    if not np.array_equal(prod(Z, y8), _exact32(_to_grid(Z, top), y8)):
        bad.append("rounding of the left operand")
    if not np.array_equal(prod(x8, Z), _exact32(x8, _to_grid(Z, top))):
        bad.append("rounding of the right operand")
    if prec == "bf16x6blk":  # both on the 16-bit grid: the six products cover every term
        x16, y16 = _on_grid(X, 16), _on_grid(Y, 16)
        if not np.array_equal(prod(x16, y16), _exact32(x16, y16)):
            bad.append("16-bit grid x 16-bit grid")
    return bad


def pins_bf16_products():
    bad = []
    prod = lambda X, Y: oracle._emu_product(X, Y, "bf16")
    g = wl.rng(34)
    Xi = g.integers(-15, 16, size=(70, 70)).astype(np.float32)
    Yi = g.integers(-15, 16, size=(70, 70)).astype(np.float32)
    if not np.array_equal(prod(Xi, Yi), _exact32(Xi, Yi)):
        bad.append("integers exact in bfloat16")
    Z = (g.standard_normal((70, 70))).astype(np.float32)
    # nearest bfloat16 by its definition: 8 significant bits, ties to even
    m, ex = np.frexp(Z.astype(np.float64))
    Zr = np.ldexp(np.rint(np.ldexp(m, 8)), ex - 8)
    if not np.array_equal(prod(Z, Yi), _exact32(Zr, Yi)):
        bad.append("rounding to bfloat16")
    return bad


def pins_integer_chain(chain, limit):
    """chain(A, n) -> (M, e) equals the exact power for every n whose powers'
    entries stay below `limit` (exact on the path's grid)."""
    bad = []
    g = wl.rng(35)
    A = g.integers(0, 2, size=(7, 7)).astype(np.float32)
    A[0, 1], A[1, 0] = 1.0, 0.0  # nonsymmetric
    for n in (2, 3, 5, 6, 7, 11, 13):
        want = oracle.matpow_value(A, n)
        if np.max(want) >= limit:
            continue
        M, e = chain(A, n)
        if not np.array_equal(np.ldexp(np.asarray(M, np.float64), e), want):
            bad.append("integer chain n=%d" % n)
    return bad


def _scalar_chain(d, n, product):
    """Right-to-left square-and-multiply of each diagonal entry with `product`."""
    out = []
    for x in d:
        p, r, bits = np.float32(x), None, int(n)
        while bits:
            if bits & 1:
                r = p if r is None else product(r, p)
            bits >>= 1
            if bits:
                p = product(p, p)
        out.append(r)
    return np.array(out, dtype=np.float64)


def pins_diagonal_chain(chain, product):
    bad = []
    d = (0.75 + 0.5 * wl.rng(36).random(40)).astype(np.float32)
    for n in (2, 3, 7, 13, 100):
        M, e = chain(np.diag(d), n)
        got = np.diag(np.ldexp(np.asarray(M, np.float64), e))
        if not np.array_equal(got, _scalar_chain(d, n, product)):
            bad.append("diagonal chain n=%d" % n)
    return bad


def pins_fp32_rounding():
    """A float32 product rounds its sums in float32: 1 + 0.75 2^-24 + 0.75 2^-24
    is 1 in float32 arithmetic and 1 + 2^-23 when summed in float64 and
    rounded once."""
    X = np.array([[1.0, 0.75 * 2 ** -24, 0.75 * 2 ** -24]] * 3, dtype=np.float32)
    Y = np.ones((3, 3), dtype=np.float32)
    got = oracle._fp32_product(X, Y)
    return [] if np.all(got == np.float32(1.0)) else ["float32 accumulation"]


f32 = lambda a, b: np.float32(np.float32(a) * np.float32(b))
bf = lambda a: np.float32(oracle.round_bf16(np.array([a], np.float32))[0])


def all_pins():
    bad = []
    for prec in ("bf16x3blk", "bf16x6blk"):
        bad += [prec + ": " + b for b in pins_block_products(prec)]
    bad += ["bf16: " + b for b in pins_bf16_products()]
    bad += ["fp32: " + b for b in pins_fp32_rounding()]
    bad += ["fp32: " + b for b in pins_integer_chain(oracle.fp32_sqmul, 2 ** 24)]
    bad += ["fp32: " + b for b in pins_diagonal_chain(oracle.fp32_sqmul, f32)]
    for prec, lim in (("bf16", 2 ** 8), ("bf16x3blk", 2 ** 16), ("bf16x6blk", 2 ** 24)):
        bad += [prec + ": " + b for b in pins_integer_chain(lambda A, n: oracle.emu_sqmul(A, n, prec), lim)]
    bad += ["bf16: " + b for b in pins_diagonal_chain(lambda A, n: oracle.emu_sqmul(A, n, "bf16"),
                                                       lambda a, b: f32(bf(a), bf(b)))]
    return bad


# ------------------------------------------------------------------ the pins hold

def test_yardstick_pins_hold():
    assert all_pins() == []


def test_grid_inputs_really_exercise_every_slice():
    # the top-grid operands need all their slices; the 8-bit ones only the first
    X = _mat(31)
    for k, top in ((2, 16), (3, 24)):
        a, _ = oracle.fixed_slices_n(_on_grid(X, top), 64, k)
        assert all(np.any(aj) for aj in a), k
        a8, _ = oracle.fixed_slices_n(_on_grid(X, 8), 64, k)
        assert np.any(a8[0]) and not any(np.any(aj) for aj in a8[1:]), k


def test_perturbation_model_scalar_closed_form():
    # 1 x 1, n = 2^K: P_0 = x (stored with its draw), P_(k+1) = P_k^2 (+draw);
    # after the power-of-two rescale each stored value is m in [0.5, 1) and the
    # draw adds rel * r, so the result is prod of (1 + rel r_k / m_k)^(2^(K-k))
    # to first order; computed here exactly in float64 from the same draws
    rel, K, x = 2.0 ** -20, 6, 0.8
    M, e = oracle.perturbed_sqmul(np.array([[x]]), 2 ** K, rel, 5)
    g = np.random.default_rng(5)
    v, E = x, 0
    for k in range(K + 1):
        f, s = math.frexp(v)
        v, E = f + rel * g.uniform(-1.0, 1.0, (1, 1))[0, 0], E + s
        if k < K:
            v = v * v
            E = 2 * E
    assert M[0, 0] * 2.0 ** e == pytest.approx(v * 2.0 ** E, rel=1e-14)


def test_perturbation_model_zero_is_the_oracle_and_is_linear():
    A = wl.gaussian(40, 3)
    M, e, _ = oracle.matpow_f64(A, 77)
    P0, f0 = oracle.perturbed_sqmul(A, 77, 0.0, 0)
    assert oracle.rel_frobenius(P0, f0, M, e) < 1e-13
    d1 = oracle.rel_frobenius(*oracle.perturbed_sqmul(A, 77, 2.0 ** -30, 1), M, e)
    d2 = oracle.rel_frobenius(*oracle.perturbed_sqmul(A, 77, 2.0 ** -29, 1), M, e)
    assert d1 > 0 and d2 / d1 == pytest.approx(2.0, rel=1e-3)
    # integer matrix, rel = 0: exact
    B = wl.fibonacci_blocks(8)
    P, f = oracle.perturbed_sqmul(B, 30, 0.0, 0)
    assert np.array_equal(np.ldexp(P, f), oracle.matpow_value(B, 30))


# ------------------------------------------------------------------ planted mistakes fail a pin

def _patched(monkeypatch, **kw):
    for name, value in kw.items():
        monkeypatch.setattr(oracle, name, value)


@pytest.mark.parametrize("prec,drop", [("bf16x3blk", (0, 1)), ("bf16x3blk", (1, 0)),
                                       ("bf16x6blk", (0, 2)), ("bf16x6blk", (2, 0)),
                                       ("bf16x6blk", (1, 1)), ("bf16x3blk", (0, 0))])
def test_planted_dropped_slice_product(monkeypatch, prec, drop):
    k, terms = oracle.SLICE_TERMS[prec]
    table = dict(oracle.SLICE_TERMS)
    table[prec] = (k, tuple(t for t in terms if t != drop))
    _patched(monkeypatch, SLICE_TERMS=table)
    assert pins_block_products(prec)


def test_planted_wrong_slice_weight(monkeypatch):
    _patched(monkeypatch, _slice_weight_exp=lambda s, j: s - 8 * (j + 1) + (1 if j == 1 else 0))
    assert pins_block_products("bf16x3blk") and pins_block_products("bf16x6blk")


def test_planted_skipped_slice_rounding(monkeypatch):
    _patched(monkeypatch, _rint=lambda u: np.asarray(u, dtype=np.float64))
    assert pins_block_products("bf16x3blk") and pins_block_products("bf16x6blk")


def test_planted_skipped_bf16_rounding(monkeypatch):
    _patched(monkeypatch, round_bf16=lambda x: np.asarray(x, dtype=np.float32))
    assert pins_bf16_products()


def test_planted_float64_accumulation(monkeypatch):
    _patched(monkeypatch, _fp32_product=lambda X, Y: _exact32(X, Y))
    assert pins_fp32_rounding()


def test_planted_transposed_operand(monkeypatch):
    orig_f, orig_e = oracle._fp32_product, oracle._emu_product
    _patched(monkeypatch, _fp32_product=lambda X, Y: orig_f(np.ascontiguousarray(X.T), Y),
             _emu_product=lambda X, Y, p: orig_e(np.ascontiguousarray(X.T), Y, p))
    assert pins_integer_chain(oracle.fp32_sqmul, 2 ** 24)
    assert pins_block_products("bf16x3blk") and pins_block_products("bf16x6blk")


def test_planted_dropped_multiply_step(monkeypatch):
    orig = oracle.schedule

    def drop_last_multiply(n):
        lv = orig(n)
        idx = [i for i, (m, _) in enumerate(lv) if m]
        if idx:
            m, s = lv[idx[-1]]
            lv[idx[-1]] = (False, s)
        return lv

    _patched(monkeypatch, schedule=drop_last_multiply)
    assert pins_integer_chain(oracle.fp32_sqmul, 2 ** 24)
    assert pins_integer_chain(lambda A, n: oracle.emu_sqmul(A, n, "bf16x6blk"), 2 ** 24)
    assert pins_diagonal_chain(oracle.fp32_sqmul, f32)
