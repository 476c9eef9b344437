"""Page-locked host buffers passed where the calls take device matrices
(GPU): the kernels read A and write the result across the host link, and
the results must equal those of device buffers bit for bit (the arithmetic
does not depend on where the input and output live)."""
import numpy as np
import pytest

import oracle
from helpers import check_float, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _pinned(x):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    return t


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("N,n", [(200, 77), (512, 1), (384, 2), (1100, 5)])
def test_f32_host_buffers_equal_device_buffers(prec, N, n):
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    A = wl.gaussian(N, N + n)
    plan = mpw.Plan(max(N, 64), prec)
    hA = _pinned(A)
    hO = torch.empty((N, N), dtype=torch.float32).pin_memory()
    hL = torch.zeros(1, dtype=torch.int64).pin_memory()
    assert all(mpw.matpow_host_accessible(t, 0) for t in (hA, hO, hL))
    mpw._check(mpw.matpow_f32(plan.h, hA, N, n, hO, hL), plan.h)
    plan.check()
    torch.cuda.synchronize()
    dO, dL = plan.f32(to_dev(A), n, mantissa=True)
    plan.check()
    assert int(hL.item()) == int(dL.item())
    assert torch.equal(hO, dO.cpu())
    M, e, _ = oracle.matpow_f64(A, n)
    err = oracle.rel_frobenius(hO.numpy(), int(hL.item()), M, e)
    check_float(err, prec, n, A, M, e, what="host buffers")
    plan.close()


def test_batched_and_mod_p_host_buffers():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    Ns, ns = [48, 130, 300, 64, 200], [9, 1, 33, 0, 1000]
    As = [wl.gaussian(k, 3 + k) for k in Ns]
    plan = mpw.Plan(max(Ns), "bf16x6")
    hA = [_pinned(a) for a in As]
    hO = [torch.empty((k, k), dtype=torch.float32).pin_memory() for k in Ns]
    hL = torch.zeros(len(Ns), dtype=torch.int64).pin_memory()
    mpw._check(mpw.matpow_batched(plan.h, hA, Ns, ns, hO, hL), plan.h)
    plan.check()
    torch.cuda.synchronize()
    dO = [torch.empty((k, k), dtype=torch.float32, device="cuda") for k in Ns]
    dL = torch.zeros(len(Ns), dtype=torch.int64, device="cuda")
    mpw._check(mpw.matpow_batched(plan.h, [to_dev(a) for a in As], Ns, ns, dO, dL), plan.h)
    plan.check()
    assert torch.equal(hL, dL.cpu())
    for h, d in zip(hO, dO):
        assert torch.equal(h, d.cpu())
    plan.close()
    # mod p, including the n = 1 copy
    N, p = 256, 65521
    A = wl.modp_uniform(N, p, 5)
    mplan = mpw.Plan(N, "fp32")
    for n in (1, 37):
        hA = torch.from_numpy(A.view(np.int32)).pin_memory()
        hO = torch.empty((N, N), dtype=torch.int32).pin_memory()
        mpw._check(mpw.matpow_mod_p(mplan.h, hA, N, n, p, hO), mplan.h)
        mplan.check()
        torch.cuda.synchronize()
        want, _ = oracle.matpow_modp(A, n, p)
        assert np.array_equal(hO.numpy().view(np.uint32), want), n
    mplan.close()


def test_host_accessible_rejects_pageable_memory():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    pageable = torch.zeros(1024, dtype=torch.float32)
    assert not mpw.matpow_host_accessible(pageable, 0)
    assert mpw.matpow_host_accessible(torch.zeros(16, device="cuda"), 0)
    assert not mpw.matpow_host_accessible(0, 0)
