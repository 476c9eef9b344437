"""Parity at the full workload sizes, in the launch configuration the bench
times, on outputs the oracle can check: the N = 8192 stochastic power
against its closed form 1 pi^T (64 sampled rows and every row sum), the
4096-matrix batch on sampled matrices against the float64 oracle, and
A^1000 mod 65521 at N = 2048 on sampled rows recomputed exactly."""
import numpy as np
import pytest

import oracle
from helpers import check_float, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_large_8192_stochastic_power_matches_closed_form():
    from paper_1204_3052_gb300 import matpow as mpw
    N, n = 8192, 2 ** 20
    A = wl.stochastic_exact(N, 0)
    plan = mpw.Plan(N, "bf16x3")
    out, lg = plan.f32(to_dev(A), n, mantissa=True)
    plan.check()
    V = np.ldexp(out.cpu().numpy().astype(np.float64), int(lg.item()))
    pi = oracle.stationary(A)
    rows = np.random.default_rng(0).choice(N, 64, replace=False)
    want = np.tile(pi, (64, 1))
    err = np.linalg.norm(V[rows] - want) / np.linalg.norm(want)
    assert err <= 2e-5 * 20, err
    assert np.max(np.abs(V.sum(axis=1) - 1.0)) <= 1e-5
    plan.close()


def test_batched_4096_sampled_against_oracle():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    bd = wl.batched_draw(count=4096, seed=0, n_max=4096)
    Ns = [int(x) for x in bd.Ns]
    ns = [int(x) for x in bd.ns]
    As = [wl.gaussian(N, int(s)) for N, s in zip(Ns, bd.seeds)]
    plan = mpw.Plan(256, "bf16x6")
    dAs = [to_dev(a) for a in As]
    outs = [torch.empty_like(a) for a in dAs]
    lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
    plan.batched(dAs, ns, outs=outs, log2=lg)
    plan.check()
    lgs = lg.cpu().numpy()
    rng = np.random.default_rng(1)
    for i in rng.choice(len(As), 48, replace=False):
        M, e, _ = oracle.matpow_f64(As[i], ns[i])
        err = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lgs[i]), M, e)
        check_float(err, "bf16x6", ns[i], As[i], M, e, what="batch 4096")
    plan.close()


def test_modp_2048_sampled_rows_exact():
    # rows of A^1000 mod p recomputed exactly: row_i(A^1000) = e_i^T A^1000 by
    # 999 vector-matrix products reduced mod p after each; every partial sum is
    # an integer below 2048 * 65520^2 < 2^43, exact in float64
    from paper_1204_3052_gb300 import matpow as mpw
    N, n, p = 2048, 1000, 65521
    A = wl.modp_uniform(N, p, 0)
    plan = mpw.Plan(N, "fp32")
    got = plan.mod_p(to_dev(A.view(np.int32)), n, p)
    plan.check()
    G = got.cpu().numpy().view(np.uint32).astype(np.uint64)
    Af = A.astype(np.float64)
    for i in (0, 777, N - 1):
        v = Af[i].copy()
        for _ in range(n - 1):
            v = np.fmod(v @ Af, p)
        assert np.array_equal(G[i], v.astype(np.uint64)), i
    plan.close()
