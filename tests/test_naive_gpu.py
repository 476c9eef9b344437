"""The comparison method (n - 1 products R <- R A, one launch each, the
paper's naive GPU method of Sec. 4.2) run with the library's product
kernels: exact where the arithmetic is exact, and within the error class of
square-and-multiply otherwise."""
import numpy as np
import pytest

import oracle
from helpers import float_tol, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def run(plan, A, n):
    dA = to_dev(A)
    out, lg = plan.f32(dA, n, mantissa=True)
    plan.check()
    return out.cpu().numpy().astype(np.float64), int(lg.item())


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
def test_naive_fibonacci_and_permutation_exact(prec):
    from paper_1204_3052_gb300 import matpow as mpw
    plan = mpw.Plan(256, prec)
    plan.set_option(mpw.OPT_NAIVE, 1)
    for N in (96, 130):
        F = wl.fibonacci_blocks(N)
        for n in (2, 3, 10, 20):
            got, ge = run(plan, F, n)
            assert np.array_equal(np.ldexp(got, ge), oracle.matpow_value(F, n)), (prec, N, n)
        P, _ = wl.permutation(N, 7)
        for n in (2, 5, 33):
            got, ge = run(plan, P, n)
            assert np.array_equal(np.ldexp(got, ge), oracle.matpow_value(P, n)), (prec, N, n)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_naive_matches_oracle_gaussian(prec):
    from paper_1204_3052_gb300 import matpow as mpw
    naive = mpw.Plan(512, prec)
    naive.set_option(mpw.OPT_NAIVE, 1)
    fast = mpw.Plan(512, prec)
    for N, n in ((100, 7), (300, 64), (512, 17)):
        A = wl.gaussian(N, N)
        M, e, _ = oracle.matpow_f64(A, n)
        gn, en = run(naive, A, n)
        gf, ef = run(fast, A, n)
        err_n = oracle.rel_frobenius(gn, en, M, e)
        err_f = oracle.rel_frobenius(gf, ef, M, e)
        # n - 1 rounded products instead of ~2 log2 n: the same error class
        assert err_n <= float_tol(n), (N, n, err_n, err_f)
    naive.close()
    fast.close()


def test_naive_launch_count():
    from paper_1204_3052_gb300 import matpow as mpw
    plan = mpw.Plan(256, "bf16x3")
    plan.set_option(mpw.OPT_NAIVE, 1)
    plan.set_option(mpw.OPT_GRAPHS, 0)
    A = to_dev(wl.gaussian(200, 1))
    before = plan.launch_count()
    plan.f32(A, 64, mantissa=True)
    plan.check()
    # one split pass + 63 products
    assert plan.launch_count() - before == 64
    plan.close()
