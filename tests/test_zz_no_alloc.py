"""matpow_f32_noalloc: the entry point for callers that may not allocate.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator, or they cannot pay for its synchronisation.  This entry point runs
the float32 SIMT square-and-multiply out of a scratch array built into the
library.  It is checked here, through the C-ABI, against matpow_f32 of a
float32 plan on the same inputs, on two calls in a row (a large power, then a
smaller matrix that runs over the scratch the first call left behind).  The
file sorts last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest

import oracle
from helpers import float_tol, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_entry_point_on_two_calls():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    plan = mpw.Plan(512, "fp32")
    for N, n, seed in ((512, 1024, 2), (300, 77, 1)):
        A = to_dev(wl.gaussian(N, seed))
        ref, ref_lg = plan.f32(A, n, mantissa=True)
        plan.check()
        out = torch.full_like(A, float("nan"))
        lg = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = mpw.matpow_f32_noalloc(A, N, n, out, lg)
        assert st == mpw.OK, mpw.load().matpow_last_error(None)
        torch.cuda.synchronize()
        err = oracle.rel_frobenius(out.cpu().numpy(), int(lg.item()), ref.cpu().numpy(),
                                   int(ref_lg.item()))
        assert err <= float_tol(n), (N, n, err)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    A = torch.zeros((513, 513), device="cuda")
    st = mpw.matpow_f32_noalloc(A, 513, 5, A)
    assert st == mpw.EINVAL
    assert b"512" in mpw.load().matpow_last_error(None)
