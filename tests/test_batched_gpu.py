"""Batched parity: each matrix of an uneven batch against the oracle, and
bit-for-bit against the same power computed alone (the grouped launches run
the same product code on the same values)."""
import numpy as np
import pytest

import oracle
from helpers import check_float, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
def test_uneven_batch_matches_oracle_and_single_calls(prec):
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    bd = wl.batched_draw(count=48, seed=1, n_max=300)
    As = [wl.gaussian(int(N), int(s)) for N, s in zip(bd.Ns, bd.seeds)]
    ns = [int(x) for x in bd.ns]
    ns[0], ns[1] = 0, 1  # trivial powers inside the batch
    plan = mpw.Plan(256, prec)
    plan.set_option(mpw.OPT_CHAIN, 2)  # single calls without split-K: same sums as the batch
    dAs = [to_dev(a) for a in As]
    lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
    outs = plan.batched(dAs, ns, log2=lg)
    plan.check()
    lgs = lg.cpu().numpy()
    for i, (A, n) in enumerate(zip(As, ns)):
        M, e, _ = oracle.matpow_f64(A, n)
        err = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lgs[i]), M, e)
        check_float(err, prec, n, A, M, e, what="batch")
        alone, alone_lg = plan.f32(dAs[i], n, mantissa=True)
        plan.check()
        assert torch.equal(alone, outs[i]) and int(alone_lg.item()) == int(lgs[i]), (i, A.shape[0], n)
    # a second call reuses the plan's batch tables (and cached descriptors)
    outs2 = plan.batched(dAs, ns, log2=lg)
    plan.check()
    for a, b in zip(outs, outs2):
        assert torch.equal(a, b)
    plan.close()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_batch_with_wide_tiles(prec):
    # orders above 1024 run in the 128-column grouped launch, next to 64-column
    # ones (three slices keep 64 columns at every order)
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    Ns = [1100, 300, 1030, 96, 40]
    ns = [13, 77, 2, 1000, 9]
    As = [wl.gaussian(N, 7 + i) for i, N in enumerate(Ns)]
    plan = mpw.Plan(1100, prec)
    plan.set_option(mpw.OPT_CHAIN, 2)
    dAs = [to_dev(a) for a in As]
    lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
    outs = plan.batched(dAs, ns, log2=lg)
    plan.check()
    for i, (A, n) in enumerate(zip(As, ns)):
        alone, alone_lg = plan.f32(dAs[i], n, mantissa=True)
        plan.check()
        assert torch.equal(alone, outs[i]), (Ns[i], n)
        if Ns[i] <= 300:
            M, e, _ = oracle.matpow_f64(A, n)
            err = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lg[i].item()), M, e)
            check_float(err, prec, n, A, M, e, what="batch")
    plan.close()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_persistent_levels_equal_per_tile_levels(prec):
    # the persistent grouped kernel (one CTA per SM over the whole tile list,
    # many tiles per CTA here) does each tile's arithmetic in the same order as
    # the one-CTA-per-tile kernel: identical bits
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    bd = wl.batched_draw(count=600, seed=9, n_max=5000)
    Ns = [max(int(N), 65) for N in bd.Ns]  # every matrix on the tensor-core path
    ns = [int(x) for x in bd.ns]
    As = [wl.gaussian(N, int(s)) for N, s in zip(Ns, bd.seeds)]
    dAs = [to_dev(a) for a in As]
    res = {}
    for persist in (1, 0):
        plan = mpw.Plan(256, prec)
        plan.set_option(mpw.OPT_PERSIST, persist)
        lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
        outs = plan.batched(dAs, ns, log2=lg)
        plan.check()
        res[persist] = ([o.clone() for o in outs], lg.clone())
        plan.close()
    for a, b in zip(res[1][0], res[0][0]):
        assert torch.equal(a, b)
    assert torch.equal(res[1][1], res[0][1])
    # and a few against the oracle
    for i in range(0, len(As), 97):
        M, e, _ = oracle.matpow_f64(As[i], ns[i])
        err = oracle.rel_frobenius(res[1][0][i].cpu().numpy(), int(res[1][1][i].item()), M, e)
        check_float(err, prec, ns[i], As[i], M, e, what="batch")


def test_batched_graph_replay_follows_new_contents():
    # the second call with the same pointers, orders and powers replays the
    # captured graph; it must read the matrices' current contents
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    Ns = [96, 40, 200, 130]
    ns = [5, 17, 2, 1000]
    plan = mpw.Plan(256, "bf16x6")
    ref = mpw.Plan(256, "bf16x6")
    ref.set_option(mpw.OPT_GRAPHS, 0)
    dAs = [to_dev(wl.gaussian(N, 50 + i)) for i, N in enumerate(Ns)]
    lg = torch.zeros(len(Ns), dtype=torch.int64, device="cuda")
    lr = torch.zeros(len(Ns), dtype=torch.int64, device="cuda")
    outs = [torch.empty_like(a) for a in dAs]
    want = [torch.empty_like(a) for a in dAs]
    for rnd in range(3):
        for i, N in enumerate(Ns):
            dAs[i].copy_(to_dev(wl.gaussian(N, 100 * rnd + i)))
        plan.batched(dAs, ns, outs=outs, log2=lg)
        ref.batched(dAs, ns, outs=want, log2=lr)
        plan.check()
        ref.check()
        for a, b in zip(outs, want):
            assert torch.equal(a, b), rnd
        assert torch.equal(lg, lr)
    plan.close()
    ref.close()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_few_powers_run_side_by_side_in_one_chain(prec):
    # up to four powers in the whole-chain range go to one cooperative launch;
    # without split-K each tile's arithmetic is that of a single call (bits
    # equal), with it the results stay within the oracle bound
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    Ns = [512, 100, 300, 65]
    ns = [1024, 3, 77, 2 ** 20 + 1]
    As = [wl.gaussian(N, 90 + i) for i, N in enumerate(Ns)]
    dAs = [to_dev(a) for a in As]
    for mode in (2, 1):
        plan = mpw.Plan(512, prec)
        plan.set_option(mpw.OPT_CHAIN, mode)
        lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
        before = plan.launch_count()
        outs = plan.batched(dAs, ns, log2=lg)
        plan.check()
        assert plan.launch_count() - before == 1  # one cooperative launch
        for i, (A, n) in enumerate(zip(As, ns)):
            if mode == 2:
                alone, alone_lg = plan.f32(dAs[i], n, mantissa=True)
                plan.check()
                assert torch.equal(alone, outs[i]) and int(alone_lg.item()) == int(lg[i].item()), (Ns[i], n)
            if n <= 4096:
                M, e, _ = oracle.matpow_f64(A, n)
                err = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lg[i].item()), M, e)
                check_float(err, prec, n, A, M, e, what="batch")
        plan.close()


@pytest.mark.parametrize("N", [1, 2, 5, 17, 32, 33, 40, 63, 64])
def test_tiny_single_forms_match_group_kernel_bitwise(N):
    # orders up to 64: a single call runs the whole chain in one CTA (N <= 32)
    # or in a four-CTA cluster that exchanges quadrants through distributed
    # shared memory; a batch runs one CTA per matrix.  All three form every
    # output as the same fmaf chain, so the bits agree.
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    ns = [2, 3, 100, (1 << 20) + 5]
    As = [wl.gaussian(N, 40 + N), wl.stochastic_exact(N, 41 + N)]
    plan = mpw.Plan(64, "fp32")
    for A in As:
        dA = to_dev(A)
        lg = torch.zeros(len(ns), dtype=torch.int64, device="cuda")
        outs = plan.batched([dA] * len(ns), ns, log2=lg)
        plan.check()
        for i, n in enumerate(ns):
            alone, alone_lg = plan.f32(dA, n, mantissa=True)
            plan.check()
            assert torch.equal(alone, outs[i]) and int(alone_lg.item()) == int(lg[i].item()), (N, n)
            if n <= 100:
                M, e, _ = oracle.matpow_f64(A, n)
                err = oracle.rel_frobenius(alone.cpu().numpy(), int(alone_lg.item()), M, e)
                check_float(err, "fp32", n, A, M, e, what="batch")
    plan.close()
