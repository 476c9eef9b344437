"""CTA-pair products (tcgen05 cta_group::2, MATPOW_OPT_PAIR) against the
one-SM kernel and the oracle (GPU).

The pair kernel computes the same exact integer slice sums and folds them
in the same order, so its results must equal the one-SM kernel's bit for bit;
the orders cover a last pair row with one valid row (N mod 256 = 1), one
whose second CTA lies wholly past row N (N mod 256 = 128), full pairs, and
levels with two products (odd powers)."""
import numpy as np
import pytest

import oracle
from helpers import check_float, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plans():
    from paper_1204_3052_gb300 import matpow as mpw
    on = mpw.Plan(4224, "bf16x3")
    on.set_option(mpw.OPT_PAIR, 1)
    off = mpw.Plan(4224, "bf16x3")
    off.set_option(mpw.OPT_PAIR, 0)
    yield on, off
    on.close()
    off.close()


@pytest.mark.parametrize("N", [2049, 2176, 2304, 3000, 4224])
def test_pair_kernel_equals_one_sm_kernel_bitwise(plans, N):
    import torch
    on, off = plans
    A = to_dev(wl.gaussian(N, N + 11))
    for n in (2, 3, 7):
        o1, l1 = on.f32(A, n, mantissa=True)
        o0, l0 = off.f32(A, n, mantissa=True)
        on.check()
        off.check()
        assert int(l1.item()) == int(l0.item()), (N, n)
        assert torch.equal(o1, o0), (N, n, (o1 - o0).abs().max().item())
    # value form too
    v1 = on.f32(A, 5)
    v0 = off.f32(A, 5)
    assert on.sync() == 0 and off.sync() == 0
    assert torch.equal(v1, v0), N


def test_pair_kernel_matches_oracle(plans):
    on, _ = plans
    N = 2304
    A = wl.gaussian(N, 5)
    for n in (2, 3):
        M, e, _ = oracle.matpow_f64(A, n)
        got, lg = on.f32(to_dev(A), n, mantissa=True)
        on.check()
        err = oracle.rel_frobenius(got.cpu().numpy(), int(lg.item()), M, e)
        check_float(err, "bf16x3", n, A, M, e, what="pair kernel")


def test_pair_kernel_exact_on_small_integers(plans):
    # integer matrices whose squares are exact: the pair's M = 256 products
    # and the fold reproduce the integer product exactly
    on, _ = plans
    g = wl.rng(77)
    for N in (2176, 2304):
        A = g.integers(-7, 8, size=(N, N)).astype(np.float32)
        got, lg = on.f32(to_dev(A), 2, mantissa=True)
        on.check()
        assert np.array_equal(np.ldexp(got.cpu().numpy().astype(np.float64), int(lg.item())),
                              oracle.gemm_f64(A, A)), N
