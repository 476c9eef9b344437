"""Pins for the CPU oracle: closed forms, invariants, brute force (CPU only).

Each test fixes the oracle against something other than itself: exact integer
arithmetic in Python, libm, the definition of the power, or an invariant of
the mathematics.  The cases are chosen so that a dropped product, a wrong
exponent bit, a transposed operand or a wrong index fails at least one test.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1204_3052_gb300 import workloads as wl


def _fib(m):
    a, b = 0, 1
    for _ in range(m):
        a, b = b, a + b
    return a


def _int_matmul(A, B, p=None):
    n = len(A)
    C = [[sum(A[i][k] * B[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    if p is not None:
        C = [[c % p for c in row] for row in C]
    return C


def _int_matpow_brute(A, n, p):
    N = len(A)
    R = [[int(i == j) % p for j in range(N)] for i in range(N)]
    for _ in range(n):
        R = _int_matmul(R, A, p)
    return R


# ---------------------------------------------------------------- products

def test_gemm_f64_exact_on_small_integers_nonsymmetric():
    # integer entries: the float64 product is exact, so it must equal Python ints.
    g = wl.rng(3)
    for N in (1, 2, 5, 7):
        A = g.integers(-50, 50, size=(N, N))
        B = g.integers(-50, 50, size=(N, N))
        ref = np.array(_int_matmul(A.tolist(), B.tolist()), dtype=np.float64)
        got = oracle.gemm_f64(A, B)
        assert np.array_equal(got, ref)  # A@B, not B@A or A^T@B


def test_gemm_modp_matches_python_ints():
    g = wl.rng(4)
    for p in (2, 7, 65521, 4294967291):
        for N in (1, 3, 8):
            A = g.integers(0, p, size=(N, N), dtype=np.uint64)
            B = g.integers(0, p, size=(N, N), dtype=np.uint64)
            ref = _int_matmul([[int(x) for x in r] for r in A], [[int(x) for x in r] for r in B], p)
            got = oracle.gemm_modp(A, B, p)
            assert got.tolist() == ref


# ---------------------------------------------------------------- schedule

@pytest.mark.parametrize("n,G", [(1, 0), (2, 1), (3, 2), (16, 4), (100, 8), (128, 7),
                                 (1024, 10), (2 ** 20, 20), (2 ** 30, 30),
                                 (2 ** 30 - 1, 29 + 29)])
def test_gemm_count_closed_form(n, G):
    # G(n) = floor(log2 n) + popcount(n) - 1
    assert oracle.gemm_count(n) == G
    assert G == (n.bit_length() - 1) + bin(n).count("1") - 1


def test_gemm_count_matches_c_oracle():
    A = wl.gaussian(3, 1)
    for n in (1, 2, 5, 6, 7, 13, 64, 100, 1000):
        _, _, g = oracle.matpow_f64(A, n, "sqmul")
        assert g == oracle.gemm_count(n)
        _, _, gb = oracle.matpow_f64(A, n, "brute")
        assert gb == n - 1


# ---------------------------------------------------------------- closed forms (float64)

@pytest.mark.parametrize("mode", ["sqmul", "brute"])
def test_fibonacci_exact(mode):
    nmax = 77 if mode == "sqmul" else 40
    for N in (2, 16, 17):
        A = wl.fibonacci_blocks(N)
        for n in range(0, nmax + 1):
            got = oracle.matpow_value(A, n, mode)
            for b in range(0, N - 1, 2):
                blk = got[b:b + 2, b:b + 2]
                want = [[_fib(n + 1), _fib(n)], [_fib(n), _fib(n - 1) if n > 0 else 1]]
                assert blk.tolist() == want, (N, n, b)
            if N % 2:
                assert got[N - 1, N - 1] == 1.0
            # off-block entries are exactly zero
            mask = np.ones((N, N), bool)
            for b in range(0, N - 1, 2):
                mask[b:b + 2, b:b + 2] = False
            if N % 2:
                mask[N - 1, N - 1] = False
            assert not np.any(got[mask])


def test_rotation_closed_form():
    for theta in (0.1, 1.0, 2.5):
        R = wl.rotation(theta)
        for n in (1, 2, 3, 7, 64, 100, 1000, 4097):
            got = oracle.matpow_value(R, n)
            want = wl.rotation(n * theta)
            assert np.max(np.abs(got - want)) <= 8 * n * 2.0 ** -52 + 1e-15, (theta, n)


def test_diagonal_matches_libm_pow():
    g = wl.rng(5)
    # entries close to 1: every d_i^n stays within float64's range relative to
    # the largest one, so each entry is checked to its own relative error.
    d = g.uniform(0.9, 1.1, size=9) * np.where(g.random(9) < 0.5, -1.0, 1.0)
    A = np.diag(d)
    for n in (1, 2, 3, 10, 77, 500, 1023):
        M, e, _ = oracle.matpow_f64(A, n)
        got = np.diag(np.ldexp(M, e))
        want = np.array([math.pow(x, n) for x in d])
        assert np.all(np.abs(got - want) <= 4 * n * 2.0 ** -52 * np.abs(want))
        off = np.ldexp(M, e) - np.diag(got)
        assert not np.any(off)


def test_diagonal_wide_range_relative_to_largest():
    # A^n shares one exponent, so entries far below the largest lose bits
    # (eventually to zero); the error is bounded relative to max|A^n|.
    g = wl.rng(5)
    d = g.uniform(0.5, 2.0, size=9) * np.where(g.random(9) < 0.5, -1.0, 1.0)
    A = np.diag(d)
    for n in (10, 500, 1023):
        M, e, _ = oracle.matpow_f64(A, n)
        want = np.array([math.pow(x, n) for x in d])
        got = np.diag(M)
        scale = np.ldexp(1.0, -e)
        assert np.all(np.abs(got - want * scale) <= 4 * n * 2.0 ** -52 * np.max(np.abs(want * scale)))


def test_diagonal_huge_exponent_keeps_range():
    # 3^(2^30) overflows float64; the mantissa/exponent form must carry it.
    A = np.diag([3.0, 0.5, 1.0])
    n = 2 ** 30
    M, e, _ = oracle.matpow_f64(A, n)
    # log2 of each diagonal entry of A^n = n*log2(d)
    l0 = math.log2(abs(M[0, 0])) + e
    assert abs(l0 - n * math.log2(3.0)) <= 1e-6 * n
    assert M[1, 1] == 0.0  # 2^-n relative to 3^n underflows the mantissa to zero


@pytest.mark.parametrize("mode", ["sqmul", "brute"])
def test_nilpotent_shift(mode):
    N = 9
    S = wl.shift(N)
    for n in range(0, 13):
        got = oracle.matpow_value(S, n, mode)
        want = np.eye(N, k=n) if n < N else np.zeros((N, N))
        assert np.array_equal(got, want), n  # superdiagonal, not subdiagonal


@pytest.mark.parametrize("mode", ["sqmul", "brute"])
def test_permutation_composed(mode):
    N = 13
    P, perm = wl.permutation(N, 7)
    idx = np.arange(N)
    for n in range(0, 30):
        got = oracle.matpow_value(P, n, mode)
        want = np.zeros((N, N))
        want[np.arange(N), idx] = 1.0
        assert np.array_equal(got, want), n
        idx = perm[idx]  # P^(n+1)[i] = perm(P^n[i])


def test_identity_and_zero_power():
    for N in (1, 4, 33):
        A = wl.gaussian(N, 2)
        assert np.array_equal(oracle.matpow_value(A, 0), np.eye(N))
        assert np.array_equal(oracle.matpow_value(np.eye(N), 12345), np.eye(N))


def test_n1_is_copy():
    A = wl.gaussian(11, 3)
    assert np.array_equal(oracle.matpow_value(A, 1), A.astype(np.float64))


def test_zero_matrix():
    A = np.zeros((5, 5), np.float32)
    assert not np.any(oracle.matpow_value(A, 7))


# ---------------------------------------------------------------- invariants

def test_power_addition_law():
    g = wl.rng(6)
    A = wl.gaussian(12, 4)
    for _ in range(6):
        m, k = int(g.integers(1, 200)), int(g.integers(1, 200))
        Mm, em, _ = oracle.matpow_f64(A, m)
        Mk, ek, _ = oracle.matpow_f64(A, k)
        prod = oracle.gemm_f64(Mm, Mk)
        Ms, es, _ = oracle.matpow_f64(A, m + k)
        assert oracle.rel_frobenius(prod, em + ek, Ms, es) <= 1e-11


@pytest.mark.parametrize("N", [2, 5, 16])
def test_brute_equals_sqmul(N):
    A = wl.gaussian(N, N)
    for n in range(1, 65):
        Ms, es, _ = oracle.matpow_f64(A, n, "sqmul")
        Mb, eb, _ = oracle.matpow_f64(A, n, "brute")
        assert oracle.rel_frobenius(Ms, es, Mb, eb) <= 1e-12 * max(n, 1)


def test_exact_stochastic_generator_rows_sum_to_one():
    for N in (1, 3, 64, 257):
        A = wl.stochastic_exact(N, 1)
        assert A.dtype == np.float32 and np.all(A >= 0)
        # float64 sum of float32 entries with a common 2^-s grid is exact
        sums = A.astype(np.float64).sum(axis=1)
        assert np.all(sums == 1.0)


def test_stochastic_row_sums_stay_one():
    A = wl.stochastic_exact(32, 0)
    for n in (2, 100, 2 ** 10, 2 ** 20):
        got = oracle.matpow_value(A, n)
        assert np.max(np.abs(got.sum(axis=1) - 1.0)) <= 1e-12


def test_stochastic_limit_is_one_pi_transpose():
    A = wl.stochastic_exact(64, 0)
    pi = oracle.stationary(A)
    want = np.outer(np.ones(64), pi)
    for n in (100, 2 ** 20):
        M, e, _ = oracle.matpow_f64(A, n)
        assert oracle.rel_frobenius(M, e, want, 0) <= 1e-12


def test_rel_frobenius_definition():
    X = np.array([[1.0, 2.0], [3.0, 4.0]])
    Y = np.array([[1.0, 2.0], [3.0, 5.0]])
    assert oracle.rel_frobenius(X, 0, Y, 0) == pytest.approx(1.0 / math.sqrt(39.0))
    # exponent alignment: X*2^3 vs (X*8)*2^0
    assert oracle.rel_frobenius(X, 3, X * 8.0, 0) == 0.0


# ---------------------------------------------------------------- mod p

@pytest.mark.parametrize("p", [2, 3, 101, 65521])
def test_modp_matches_python_bruteforce(p):
    g = wl.rng(p)
    for N in (1, 2, 4, 8):
        A = g.integers(0, p, size=(N, N), dtype=np.uint64)
        Ai = [[int(x) for x in r] for r in A]
        for n in (0, 1, 2, 3, 17, 64, 129, 200):
            got, _ = oracle.matpow_modp(A, n, p)
            assert got.tolist() == _int_matpow_brute(Ai, n, p), (p, N, n)


def test_modp_fibonacci_huge_power():
    p = 65521
    A = wl.fibonacci_blocks(4).astype(np.uint64)
    for n in (10 ** 6, 2 ** 30, 2 ** 30 - 1, 123456789):
        got, _ = oracle.matpow_modp(A, n, p)
        # Python's pow on the 2x2 Fibonacci matrix by a separate exact method:
        # fast doubling F(2k) = F(k)(2F(k+1) - F(k)), F(2k+1) = F(k)^2 + F(k+1)^2
        def fd(m):
            if m == 0:
                return (0, 1)
            a, b = fd(m // 2)
            c = (a * ((2 * b - a) % p)) % p
            d = (a * a + b * b) % p
            return (d, (c + d) % p) if m % 2 else (c, d)
        Fn, Fn1 = fd(n)
        Fnm1 = (Fn1 - Fn) % p
        assert got[:2, :2].tolist() == [[Fn1, Fn], [Fn, Fnm1]]
        assert got[2:, 2:].tolist() == [[Fn1, Fn], [Fn, Fnm1]]


def test_modp_diagonal_matches_pow():
    p = 65521
    d = [2, 3, 65520, 12345, 0, 1]
    A = np.diag(np.array(d, dtype=np.uint64))
    for n in (1, 5, 2 ** 30, 999999937):
        got, _ = oracle.matpow_modp(A, n, p)
        assert np.diag(got).tolist() == [pow(x, n, p) for x in d]


def test_modp_power_of_power():
    p = 65521
    A = wl.modp_uniform(6, p, 9).astype(np.uint64)
    for m, k in ((3, 5), (7, 11), (64, 2)):
        Am, _ = oracle.matpow_modp(A, m, p)
        Amk, _ = oracle.matpow_modp(Am, k, p)
        direct, _ = oracle.matpow_modp(A, m * k, p)
        assert np.array_equal(Amk, direct)


def test_modp_brute_equals_sqmul():
    p = 65521
    A = wl.modp_uniform(16, p, 1).astype(np.uint64)
    for n in range(0, 65):
        s, _ = oracle.matpow_modp(A, n, p, "sqmul")
        b, _ = oracle.matpow_modp(A, n, p, "brute")
        assert np.array_equal(s, b), n


def test_modp_rejects_unreduced_entries():
    A = np.array([[5, 1], [0, 2]], dtype=np.uint64)
    with pytest.raises(RuntimeError):
        oracle.matpow_modp(A, 3, 5)


# ---------------------------------------------------------------- precision emulators

def test_round_bf16_known_values():
    # bfloat16 has 8 significant bits: spacing 2^-7 in [1, 2)
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, 1.0 + 2 ** -9,
                  -(1.0 + 3 * 2 ** -8), 3.0, 0.0, 2 ** -100, 65280.0, 65408.0], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, 1.0,
                     -(1.0 + 2 ** -6), 3.0, 0.0, 2 ** -100, 65280.0, 65536.0], dtype=np.float32)
    assert np.array_equal(oracle.round_bf16(x), want)


def test_round_bf16_is_nearest():
    g = wl.rng(11)
    x = g.standard_normal(20000).astype(np.float32)
    r = oracle.round_bf16(x).astype(np.float64)
    # every bf16 value has 7 fraction bits: r * 2^(7 - exponent) is an integer
    m, e = np.frexp(r)
    assert np.all(m * 256 == np.round(m * 256))
    # nearest: |x - r| <= half a bf16 ulp of x
    _, ex = np.frexp(x.astype(np.float64))
    assert np.all(np.abs(x - r) <= np.ldexp(1.0, ex - 9) + 0.0)


def test_split_bf16_sixteen_bits_exact():
    # values with at most 16 significant bits are hi + lo exactly
    g = wl.rng(12)
    ints = g.integers(-(2 ** 15), 2 ** 15, size=5000).astype(np.float64)
    x = np.ldexp(ints, g.integers(-20, 20, size=5000)).astype(np.float32)
    hi, lo = oracle.split_bf16(x)
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), x.astype(np.float64))
    # and a general float32 keeps ~16 bits: |x - hi - lo| <= 2^-16 |x|
    y = g.standard_normal(5000).astype(np.float32)
    h, l = oracle.split_bf16(y)
    assert np.all(np.abs(y.astype(np.float64) - h - l) <= 2.0 ** -16 * np.abs(y))


def test_emulated_paths_are_exact_on_small_integers():
    # Fibonacci powers stay integers below 2^8 for n <= 12: every operand is
    # exact in bfloat16, so both emulated precisions reproduce the power exactly
    A = wl.fibonacci_blocks(6)
    for prec in ("bf16", "bf16x3"):
        for n in range(1, 12):
            M, e = oracle.emu_sqmul(A, n, prec)
            assert np.array_equal(np.ldexp(M.astype(np.float64), e), oracle.matpow_value(A, n))


def test_emulated_error_ordering():
    # bf16 error > bf16x3 error > float32 error on a Gaussian power
    A = wl.gaussian(64, 1)
    n = 16
    M, e, _ = oracle.matpow_f64(A, n)
    errs = {}
    for prec in ("bf16", "bf16x3"):
        Mp, ep = oracle.emu_sqmul(A, n, prec)
        errs[prec] = oracle.rel_frobenius(Mp, ep, M, e)
    Mf, ef = oracle.fp32_sqmul(A, n)
    errs["fp32"] = oracle.rel_frobenius(Mf, ef, M, e)
    assert errs["bf16"] > 30 * errs["bf16x3"]
    assert errs["bf16x3"] > errs["fp32"]
    assert errs["bf16"] < 2.0 ** -6


def test_fixed_slices_integers_and_reconstruction():
    g = wl.rng(13)
    X = (g.standard_normal((40, 40)) * 3.0).astype(np.float32)
    a1, a2, s = oracle.fixed_slices(X)
    assert np.all(a1 == np.rint(a1)) and np.all(a2 == np.rint(a2))
    assert np.max(np.abs(a1)) <= 256 and np.max(np.abs(a2)) <= 128
    # max|X| * 2^-s in [0.5, 1)
    assert 0.5 <= np.max(np.abs(X)) * 2.0 ** -s < 1.0
    rec = np.ldexp(256.0 * a1 + a2, s - 16)
    assert np.max(np.abs(rec - X)) <= 2.0 ** (s - 17)
    # values on the 2^(s-16) grid are reproduced exactly
    Y = np.ldexp(np.rint(np.ldexp(X.astype(np.float64), 16 - s)), s - 16).astype(np.float32)
    b1, b2, t = oracle.fixed_slices(Y)
    assert t == s and np.array_equal(np.ldexp(256.0 * b1 + b2, t - 16), Y.astype(np.float64))


def test_fixed_slice_products_stay_exact_in_float32():
    # |a1 b1| <= 2^16 and |a1 b2 + a2 b1| <= 2^16, so 256-deep sums stay <= 2^24
    assert 256 * 256 * 256 <= 2 ** 24
    assert 256 * (256 * 128 + 128 * 256) <= 2 ** 24


def test_emulated_fixed_split_close_to_float_split():
    A = wl.gaussian(96, 2)
    n = 16
    M, e, _ = oracle.matpow_f64(A, n)
    Mx, ex = oracle.emu_sqmul(A, n, "bf16x3fx")
    Mh, eh = oracle.emu_sqmul(A, n, "bf16x3")
    efx = oracle.rel_frobenius(Mx, ex, M, e)
    efl = oracle.rel_frobenius(Mh, eh, M, e)
    # 16-bit fixed point relative to the matrix maximum keeps fewer bits of
    # the small entries than a per-entry 16-bit split: larger, but bounded
    assert efl < efx < 30 * efl and efx < 1e-3


def test_block_fixed_slices_reconstruct_per_block():
    g = wl.rng(14)
    X = (g.standard_normal((130, 130)) * np.exp(g.standard_normal((130, 130)))).astype(np.float32)
    a1, a2, s = oracle.fixed_slices(X, 64)
    assert np.all(np.abs(a1) <= 256) and np.all(np.abs(a2) <= 128)
    rec = np.ldexp(256.0 * a1 + a2, s - 16)
    assert np.all(np.abs(rec - X) <= np.ldexp(1.0, s - 17))
    # each tile's own maximum sets its exponent
    for i in range(0, 130, 64):
        for j in range(0, 130, 64):
            t = np.abs(X[i:i + 64, j:j + 64]).max()
            assert 0.5 <= t * 2.0 ** -s[i, j] < 1.0
    # the block emulator agrees with the global one when one block covers the matrix
    A = wl.gaussian(60, 3)
    Mb, eb = oracle.emu_sqmul(A, 9, "bf16x3blk")
    Mg, eg = oracle.emu_sqmul(A, 9, "bf16x3fx")
    assert oracle.rel_frobenius(Mb, eb, Mg, eg) < 1e-6


def test_three_slices_integers_and_top_binade_exact():
    g = wl.rng(15)
    X = (g.standard_normal((130, 130)) * np.exp(g.standard_normal((130, 130)))).astype(np.float32)
    a, s = oracle.fixed_slices_n(X, 64, 3)
    assert len(a) == 3
    assert all(np.all(aj == np.rint(aj)) for aj in a)
    assert np.all(np.abs(a[0]) <= 256) and np.all(np.abs(a[1]) <= 128) and np.all(np.abs(a[2]) <= 128)
    # the first two slices are the two-slice split
    b1, b2, t = oracle.fixed_slices(X, 64)
    assert np.array_equal(a[0], b1) and np.array_equal(a[1], b2) and np.array_equal(s, t)
    rec = np.ldexp(65536.0 * a[0] + 256.0 * a[1] + a[2], s - 24)
    assert np.all(np.abs(rec - X) <= np.ldexp(1.0, s - 25))
    # float32 entries in their block's top binade sit on the 2^(s-24) grid: exact
    top = np.abs(X) >= np.ldexp(1.0, s - 1)
    assert top.sum() >= 4 and np.array_equal(rec[top], X[top].astype(np.float64))


def test_six_products_exact_on_sixteen_bit_grid():
    # Entries on each block's 2^(s-16) grid have a third slice of zero, so the
    # six products a_i b_j (i + j <= 2) cover every nonzero term: the emulated
    # product is the exact product rounded once to float32 (a dropped a1 b1,
    # a wrong slice weight or a transposed operand all break this).
    g = wl.rng(16)
    def grid16(X):
        _, _, s = oracle.fixed_slices(X, 64)
        return np.ldexp(np.rint(np.ldexp(X.astype(np.float64), 16 - s)), s - 16).astype(np.float32)
    X = grid16((g.standard_normal((100, 100)) * np.exp(g.standard_normal((100, 100)))).astype(np.float32))
    Y = grid16((g.standard_normal((100, 100)) * np.exp(g.standard_normal((100, 100)))).astype(np.float32))
    a, _ = oracle.fixed_slices_n(X, 64, 3)
    assert not np.any(a[2])
    exact = (X.astype(np.float64) @ Y.astype(np.float64)).astype(np.float32)
    assert np.array_equal(oracle._emu_product(X, Y, "bf16x6blk"), exact)
    # the two-slice emulator drops a1 b1 there and differs
    assert not np.array_equal(oracle._emu_product(X, Y, "bf16x3blk"), exact)


def test_six_product_chain_at_float32_accuracy():
    A = wl.gaussian(96, 2)
    for n in (16, 1000):
        M, e, _ = oracle.matpow_f64(A, n)
        e6 = oracle.rel_frobenius(*oracle.emu_sqmul(A, n, "bf16x6blk"), M, e)
        e3 = oracle.rel_frobenius(*oracle.emu_sqmul(A, n, "bf16x3blk"), M, e)
        ef = oracle.rel_frobenius(*oracle.fp32_sqmul(A, n), M, e)
        # 24-bit fixed point per block: float32-class, far below two slices
        assert e6 < 3 * ef and e6 * 50 < e3
