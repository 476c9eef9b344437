"""Mod-p parity: libmatpow (GPU) against the exact uint64 CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from helpers import to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["tensor", "simt"])
def plan(request):
    from paper_1204_3052_gb300 import matpow as mpw
    p = mpw.Plan(1024, "bf16x3")
    p.set_option(mpw.OPT_MODP_TC, 1 if request.param == "tensor" else 0)
    yield p
    p.close()


def run(plan, A, n, p):
    dA = to_dev(A.astype(np.uint32).view(np.int32))
    out = plan.mod_p(dA, n, p)
    st = plan.sync()
    return out.cpu().numpy().view(np.uint32).astype(np.uint64), st


@pytest.mark.parametrize("N", [1, 2, 3, 8, 17, 64, 65, 100, 129, 256, 300])
def test_modp_random_bit_exact(plan, N):
    p = 65521
    A = wl.modp_uniform(N, p, N)
    for n in (0, 1, 2, 3, 100, 2 ** 20, 2 ** 30 - 1):
        got, st = run(plan, A, n, p)
        want, _ = oracle.matpow_modp(A, n, p)
        assert st == 0
        assert np.array_equal(got, want), (N, n)


@pytest.mark.parametrize("p", [2, 3, 251, 257, 65521, 65536])
def test_modp_moduli(plan, p):
    A = wl.modp_uniform(40, p, 3)
    for n in (5, 999):
        got, st = run(plan, A, n, p)
        want, _ = oracle.matpow_modp(A, n, p)
        assert st == 0 and np.array_equal(got, want), (p, n)


def test_modp_fibonacci_huge(plan):
    p = 65521
    A = wl.fibonacci_blocks(64).astype(np.uint64)
    n = 10 ** 18 + 7
    got, st = run(plan, A, n, p)
    want, _ = oracle.matpow_modp(A, n, p)
    assert np.array_equal(got, want)


def test_modp_rejects_unreduced(plan):
    A = wl.modp_uniform(10, 7, 1)
    A[3, 4] = 7
    got, st = run(plan, A, 5, 7)
    assert st == 1  # MATPOW_EINVAL from the device check


def test_modp_tensor_and_simt_agree_on_large_orders():
    from paper_1204_3052_gb300 import matpow as mpw
    import torch
    tc = mpw.Plan(2100, "fp32")
    sm = mpw.Plan(2100, "fp32")
    sm.set_option(mpw.OPT_MODP_TC, 0)
    for N, n, p in ((1000, 77, 65521), (2100, 5, 65536), (513, 2 ** 40 + 3, 251)):
        A = wl.modp_uniform(N, p, N)
        dA = to_dev(A.view(np.int32))
        a = tc.mod_p(dA, n, p)
        b = sm.mod_p(dA, n, p)
        assert tc.sync() == 0 and sm.sync() == 0
        assert torch.equal(a, b), (N, n, p)
    tc.close()
    sm.close()


def test_walk_counts_mod_p(plan):
    # graph walk counting: (A^n)[i, j] is the number of walks of length n from
    # i to j in the graph with 0/1 adjacency A; counted here by dynamic
    # programming over walk lengths with Python integers (exact, independent
    # of the oracle), then reduced mod p
    p = 65521
    g = wl.rng(31)
    for N, n in ((70, 9), (130, 25)):
        A = (g.random((N, N)) < 0.1).astype(np.uint64)
        src = [0, N // 2, N - 1]
        got, st = run(plan, A, n, p)
        assert st == 0
        adj = [[j for j in range(N) if A[i, j]] for i in range(N)]
        for s in src:
            walks = [0] * N
            walks[s] = 1
            for _ in range(n):
                nxt = [0] * N
                for i, w in enumerate(walks):
                    if w:
                        for j in adj[i]:
                            nxt[j] += w
                walks = nxt
            assert [int(v) for v in got[s]] == [w % p for w in walks], (N, n, s)
