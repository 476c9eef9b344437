"""Batched parity: each matrix of an uneven batch against the oracle."""
import numpy as np
import pytest

import oracle
from helpers import gate, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32"])
def test_uneven_batch_matches_single_calls(prec):
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    bd = wl.batched_draw(count=48, seed=1, n_max=300)
    As = [wl.gaussian(int(N), int(s)) for N, s in zip(bd.Ns, bd.seeds)]
    ns = [int(x) for x in bd.ns]
    ns[0], ns[1] = 0, 1  # trivial powers inside the batch
    plan = mpw.Plan(256, prec)
    dAs = [to_dev(a) for a in As]
    lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
    outs = plan.batched(dAs, ns, log2=lg)
    plan.check()
    lgs = lg.cpu().numpy()
    for i, (A, n) in enumerate(zip(As, ns)):
        M, e, _ = oracle.matpow_f64(A, n)
        err = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lgs[i]), M, e)
        Mf, ef = oracle.fp32_sqmul(A, n)
        assert err <= gate(n, oracle.rel_frobenius(Mf, ef, M, e)), (i, A.shape[0], n, err)
    # a second call reuses the plan's batch tables
    outs2 = plan.batched(dAs, ns, log2=lg)
    plan.check()
    for a, b in zip(outs, outs2):
        assert torch.equal(a, b)
    plan.close()
