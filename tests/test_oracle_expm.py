"""Pins of the oracle's matrix exponential (CPU only): closed forms, group
identities and an independent library routine.  A dropped series term, a
wrong factorial, a wrong scaling exponent or a transposed product fails one
of these."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def rel(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


@pytest.mark.parametrize("scale", [0.1, 1.0, 6.0])
def test_diagonal_is_elementwise_exp(scale):
    d = np.linspace(-1.0, 1.0, 9) * scale
    E = oracle.expm_f64(np.diag(d))
    assert rel(np.diag(E), np.array([math.exp(x) for x in d])) < 1e-14
    assert np.count_nonzero(E - np.diag(np.diag(E))) == 0


def test_nilpotent_series_is_exact_polynomial():
    # strictly upper triangular integer N: e^N = sum_{k < 6} N^k / k! exactly
    rng = np.random.default_rng(5)
    Nm = np.triu(rng.integers(-3, 4, (6, 6)), 1)
    Nf = [[Fraction(int(v)) for v in row] for row in Nm]

    def mul(X, Y):
        return [[sum(X[i][k] * Y[k][j] for k in range(6)) for j in range(6)] for i in range(6)]

    P = [[Fraction(int(i == j)) for j in range(6)] for i in range(6)]
    S = [row[:] for row in P]
    for k in range(1, 6):
        P = mul(P, Nf)
        S = [[S[i][j] + P[i][j] / math.factorial(k) for j in range(6)] for i in range(6)]
    want = np.array([[float(v) for v in row] for row in S])
    assert rel(oracle.expm_f64(Nm.astype(np.float64)), want) < 1e-14


@pytest.mark.parametrize("theta", [0.3, 2.0, 10.0])
def test_rotation_generator(theta):
    # e^(theta J), J = [[0, -1], [1, 0]]: the rotation by theta (block diagonal x3)
    J = np.array([[0.0, -1.0], [1.0, 0.0]])
    A = np.kron(np.eye(3), theta * J)
    R = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    assert rel(oracle.expm_f64(A), np.kron(np.eye(3), R)) < 1e-13


def test_jordan_block():
    # e^(lambda I + N) = e^lambda (I + N + N^2/2 + N^3/6) for the 4x4 shift N
    lam = -0.7
    Nm = np.eye(4, k=1)
    want = math.exp(lam) * (np.eye(4) + Nm + Nm @ Nm / 2 + Nm @ Nm @ Nm / 6)
    assert rel(oracle.expm_f64(lam * np.eye(4) + Nm), want) < 1e-14


def test_group_identities():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((16, 16)) * 0.6
    E = oracle.expm_f64(A)
    assert rel(oracle.gemm_f64(E, oracle.expm_f64(-A)), np.eye(16)) < 1e-12
    assert rel(oracle.expm_f64(2 * A), oracle.gemm_f64(E, E)) < 1e-12
    assert rel(oracle.expm_f64(A + 0.5 * np.eye(16)), math.exp(0.5) * E) < 1e-13


def test_scaling_exponent():
    A = np.zeros((3, 3))
    A[0, 1] = 5.0  # ||A||_1 = 5
    assert oracle.expm_scaling(A, 0.5) == 4  # 5 / 16 <= 1/2 < 5 / 8
    assert oracle.expm_scaling(A, 1.0) == 3
    assert oracle.expm_scaling(np.eye(3) * 0.25, 0.5) == 0


@pytest.mark.parametrize("scale", [0.05, 1.0, 8.0])
def test_matches_independent_pade_routine(scale):
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(int(scale * 100))
    A = rng.standard_normal((24, 24)) * scale / math.sqrt(24)
    assert rel(oracle.expm_f64(A), sl.expm(A)) < 1e-13


def test_fp32_yardstick_is_float32_class():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((32, 32)) * 2.0 / math.sqrt(32)
    M, e = oracle.expm_fp32_ps(A)
    err = rel(np.ldexp(M.astype(np.float64), e), oracle.expm_f64(A))
    assert 1e-9 < err < 1e-5
