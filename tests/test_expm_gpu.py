"""Parity of matpow_expm (e^A by scaling and squaring on the product and
squaring kernels) against the float64 oracle, on the small-order path
(N <= 64), the whole-chain range and the level path, plus the edge cases."""
import math

import numpy as np
import pytest

import oracle
from helpers import to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def gate(A, want):
    """The stated bound 2e-5 (s + 1) for float32-class results (FP32 SIMT and
    BF16X6 products; every order up to 64, which runs the float32 path) and s."""
    s = oracle.expm_scaling(A, 1.0)
    return 2e-5 * (s + 1), s


def split_gate(A, want):
    """BF16X3 (16-bit slices): max(stated, 2 x the error of the same
    evaluation with the split's operand rounding emulated on the CPU)."""
    g, s = gate(A, want)
    if A.shape[0] > 64:
        M, e = oracle.expm_emu_ps(A, "bf16x3blk")
        emu = np.linalg.norm(np.ldexp(M.astype(np.float64), e) - want) / np.linalg.norm(want)
        g = max(g, 2.0 * emu)
    return g, s


_cache = {}


def case(N, scale):
    """Input, oracle e^A and gate for one (N, scale), computed once."""
    if (N, scale) not in _cache:
        A = (wl.gaussian(N, 60 + N) * scale).astype(np.float32)
        want = oracle.expm_f64(A)
        _cache[(N, scale)] = (A, want) + gate(A, want)
    return _cache[(N, scale)]


@pytest.fixture(scope="module")
def plans():
    from paper_1204_3052_gb300 import matpow as mpw
    ps = {prec: mpw.Plan(700, prec) for prec in ("fp32", "bf16x6", "bf16x3")}
    yield ps
    for p in ps.values():
        p.close()


def run(plan, A):
    out, lg = plan.expm(to_dev(A), mantissa=True)
    plan.check()
    return np.ldexp(out.cpu().numpy().astype(np.float64), int(lg.item()))


CASES = [(N, sc) for N in (1, 5, 33, 64, 65, 130, 300) for sc in (0.05, 1.0, 4.0)] + [(700, 1.0)]


@pytest.mark.parametrize("N,scale", CASES)
@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_expm_gaussian_matches_oracle(plans, prec, N, scale):
    A, want, g, s = case(N, scale)
    got = run(plans[prec], A)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print("e^A prec=%s N=%d s=%d rel_F=%.3e bound=%.3e [stated]" % (prec, N, s, err, g))
    assert err <= g, (prec, N, scale, s, err, g)


@pytest.mark.parametrize("N", [40, 200])
def test_expm_bf16x3_is_within_its_split_error(plans, N):
    # two slices keep 16 bits relative to a block maximum (orders above 64;
    # up to 64 the float32 path runs): gate on the same evaluation emulated
    A = (wl.gaussian(N, 7) * 2.0).astype(np.float32)
    want = oracle.expm_f64(A)
    got = run(plans["bf16x3"], A)
    g, s = split_gate(A, want)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print("e^A bf16x3 N=%d s=%d rel_F=%.3e bound=%.3e" % (N, s, err, g))
    assert err <= g, (N, s, err, g)


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_expm_closed_forms(plans, prec):
    from paper_1204_3052_gb300 import matpow as mpw
    p = plans[prec]
    for N in (20, 100):
        # zero -> identity exactly
        assert np.array_equal(run(p, np.zeros((N, N), np.float32)), np.eye(N))
        # diagonal -> elementwise exp
        d = np.linspace(-3.0, 3.0, N).astype(np.float32)
        got = run(p, np.diag(d))
        assert np.max(np.abs(np.diag(got) / np.exp(d.astype(np.float64)) - 1.0)) < 2e-5 * 4
        assert np.count_nonzero(got - np.diag(np.diag(got))) == 0
    # beyond float32: e^(100 I + G) in the mantissa form; value mode -> inf and ERANGE
    A = (100.0 * np.eye(80) + wl.gaussian(80, 2) * 0.5).astype(np.float32)
    want = math.exp(100.0) * oracle.expm_f64(A - 100.0 * np.eye(80, dtype=np.float32))
    got = run(p, A)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5 * 9
    val = p.expm(to_dev(A))
    assert p.sync() == mpw.ERANGE
    assert np.all(np.isinf(np.diag(val.cpu().numpy())))


def test_expm_edge_cases(plans):
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    p = plans["bf16x6"]
    A = (wl.gaussian(96, 4) * 2.0).astype(np.float32)
    # dOut may alias dA
    dA = to_dev(A)
    lg = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert mpw.matpow_expm(p.h, dA, 96, dA, lg) == mpw.OK
    p.check()
    got = np.ldexp(dA.cpu().numpy().astype(np.float64), int(lg.item()))
    want = oracle.expm_f64(A)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= gate(A, want)[0]
    # non-finite input: rejected after the norm read-back
    bad = A.copy()
    bad[3, 5] = np.nan
    out = torch.empty_like(dA)
    assert mpw.matpow_expm(p.h, to_dev(bad), 96, out, None) == mpw.EINVAL
    # empty matrix and too large an order
    assert mpw.matpow_expm(p.h, dA, 0, out, None) == mpw.OK
    assert mpw.matpow_expm(p.h, dA, 701, out, None) == mpw.EINVAL
    assert p.sync() == mpw.OK


def test_expm_other_paths():
    # plain BF16 products (8 significant bits: a loose class) and the
    # tensor-core path at N = 64 (tiny_max = 0: one 64 x 64 block, one tile)
    from paper_1204_3052_gb300 import matpow as mpw
    A = (wl.gaussian(100, 9) * 1.5).astype(np.float32)
    want = oracle.expm_f64(A)
    p = mpw.Plan(128, "bf16")
    err = np.linalg.norm(run(p, A) - want) / np.linalg.norm(want)
    p.close()
    assert err < 0.1, err
    p = mpw.Plan(64, "bf16x6")
    p.set_option(mpw.OPT_TINY_MAX, 0)
    for N in (64,):
        A = (wl.gaussian(N, 10 + N) * 2.0).astype(np.float32)
        want = oracle.expm_f64(A)
        g, s = gate(A, want)
        err = np.linalg.norm(run(p, A) - want) / np.linalg.norm(want)
        assert err <= g, (N, s, err, g)
    p.close()


def test_expm_refuses_stream_capture():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    p = mpw.Plan(128, "bf16x6")
    A = to_dev((wl.gaussian(96, 4)).astype(np.float32))
    out = torch.empty_like(A)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        st = mpw.matpow_expm(p.h, A, 96, out, None, s)
        g.capture_end()
    assert st == mpw.EINVAL
    assert "captured" in mpw.load().matpow_last_error(p.h).decode()
    assert p.sync() == mpw.OK
    p.close()


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3"])
def test_expm_bench_workload(plans, prec):
    # the bench's e^A input (4 N(0, 1/N) of order 512, seed 0; s = 7) through
    # the same call the bench times
    A = (wl.gaussian(512, 0) * 4.0).astype(np.float32)
    want = oracle.expm_f64(A)
    g, s = split_gate(A, want) if prec == "bf16x3" else gate(A, want)
    assert s == 7
    err = np.linalg.norm(run(plans[prec], A) - want) / np.linalg.norm(want)
    print("e^A bench prec=%s rel_F=%.3e bound=%.3e" % (prec, err, g))
    assert err <= g, (prec, err, g)
