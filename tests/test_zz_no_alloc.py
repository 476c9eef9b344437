"""matpow_f32_noalloc: the entry point for callers that may not allocate.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator, or they cannot pay for its synchronisation.  This entry point runs
the float32 SIMT square-and-multiply out of a scratch array built into the
library.  It is checked here, through the C-ABI, against the float64 oracle
and against matpow_f32 of a float32 plan on the same inputs, on two calls in a
row (a large power, then a smaller matrix that runs over the scratch the first
call left behind), and on small orders, n = 0 and n = 1, in value and
mantissa form.  The file sorts last so that a failure here cannot hide any
other test.
"""
import numpy as np
import pytest

import oracle
from helpers import check_float, float_tol, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_matches_oracle_and_plan_entry_point_on_two_calls():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    plan = mpw.Plan(512, "fp32")
    for N, n, seed in ((512, 1024, 2), (300, 77, 1)):
        A_host = wl.gaussian(N, seed)
        A = to_dev(A_host)
        ref, ref_lg = plan.f32(A, n, mantissa=True)
        plan.check()
        out = torch.full_like(A, float("nan"))
        lg = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = mpw.matpow_f32_noalloc(A, N, n, out, lg)
        assert st == mpw.OK, mpw.load().matpow_last_error(None)
        torch.cuda.synchronize()
        M, e, _ = oracle.matpow_f64(A_host, n)
        err = oracle.rel_frobenius(out.cpu().numpy(), int(lg.item()), M, e)
        check_float(err, "fp32", n, A_host, M, e, what="no-alloc")
        d = oracle.rel_frobenius(out.cpu().numpy(), int(lg.item()), ref.cpu().numpy(), int(ref_lg.item()))
        assert d <= float_tol(n), (N, n, d)
    plan.close()


@pytest.mark.parametrize("N", [1, 17, 64])
def test_noalloc_small_orders_both_forms(N):
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    A_host = wl.gaussian(N, 40 + N)
    A = to_dev(A_host)
    for n in (0, 1, 2, 3, 1000):
        M, e, _ = oracle.matpow_f64(A_host, n)
        want = np.ldexp(M, e)
        out = torch.full_like(A, float("nan"))
        lg = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert mpw.matpow_f32_noalloc(A, N, n, out, lg) == mpw.OK
        torch.cuda.synchronize()
        M_gpu, e_gpu = out.cpu().numpy().astype(np.float64), int(lg.item())
        mant = np.ldexp(M_gpu, e_gpu)
        val = torch.full_like(A, float("nan"))
        assert mpw.matpow_f32_noalloc(A, N, n, val, None) == mpw.OK
        torch.cuda.synchronize()
        val = val.cpu().numpy().astype(np.float64)
        if n <= 1:  # the identity and a copy: exact
            assert np.array_equal(mant, want) and np.array_equal(val, want), (N, n)
            continue
        # exponents aligned first: A^1000 of these inputs lies outside float64 too
        err = oracle.rel_frobenius(M_gpu, e_gpu, M, e)
        check_float(err, "fp32", n, A_host, M, e, what="no-alloc N=%d" % N)
        # value form: the mantissa form rescaled in float64 and rounded once to
        # float32 (0 or +-inf where the power leaves the float32 range)
        with np.errstate(over="ignore", under="ignore"):
            assert np.array_equal(val, mant.astype(np.float32).astype(np.float64)), (N, n)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    A = torch.zeros((513, 513), device="cuda")
    st = mpw.matpow_f32_noalloc(A, 513, 5, A)
    assert st == mpw.EINVAL
    assert b"512" in mpw.load().matpow_last_error(None)
