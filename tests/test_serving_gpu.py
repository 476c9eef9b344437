"""Serving: continuous batching gives every request the result it gets alone.

Requests of mixed order, power and kind are submitted in bursts while earlier
ones run, so each scheduler step mixes requests at different levels.  Each
float result must equal, bit for bit, the same power computed alone through
matpow_f32 (the grouped launch runs the same product code on the same
values), and must match the oracle; mod-p results must equal the oracle
exactly.
"""
import time

import numpy as np
import pytest

import oracle
from helpers import check_float, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def make_requests(count, seed):
    g = wl.rng(seed)
    reqs = []
    for i in range(count):
        kind = 1 if g.random() < 0.2 else 0
        N = int(wl.log_uniform_int(g, 8, 300, 1)[0])
        n = int(g.choice([0, 1, 2, 3, 5, 17, 64, 100, 255, 1000, 2 ** 20 + 3]))
        A = wl.modp_uniform(N, 65521, 100 + i) if kind else wl.gaussian(N, 100 + i)
        reqs.append((kind, N, n, A))
    return reqs


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
def test_mixed_stream_matches_isolated_runs(prec):
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    server = mpw.Server(300, prec, hbm_budget_bytes=64 << 20, max_inflight=12)
    plan = mpw.Plan(300, prec)
    plan.set_option(mpw.OPT_CHAIN, 2)  # isolated runs without split-K: same sums as the server
    reqs = make_requests(60, 5)
    dev = []
    tickets = []
    for i, (kind, N, n, A) in enumerate(reqs):
        if kind:
            dA = to_dev(A.view(np.int32))
            out = torch.empty_like(dA)
            lg = None
            t = server.submit(dA, n, out, kind=1, p=65521)
        else:
            dA = to_dev(A)
            out = torch.empty_like(dA)
            lg = torch.zeros(1, dtype=torch.int64, device="cuda")
            t = server.submit(dA, n, out, log2_scale=lg)
        dev.append((dA, out, lg))
        tickets.append(t)
        if i % 7 == 6:
            time.sleep(0.002)  # later requests arrive while earlier ones run
    for t in tickets:
        assert server.wait(t) == mpw.OK
    torch.cuda.synchronize()
    for (kind, N, n, A), (dA, out, lg) in zip(reqs, dev):
        if kind:
            want, _ = oracle.matpow_modp(A, n, 65521)
            got = out.cpu().numpy().view(np.uint32).astype(np.uint64)
            assert np.array_equal(got, want), (N, n)
            continue
        alone, alone_lg = plan.f32(dA, n, mantissa=True)
        plan.check()
        assert torch.equal(out, alone) and int(lg.item()) == int(alone_lg.item()), (N, n)
        if n <= 1000:
            M, e, _ = oracle.matpow_f64(A, n)
            err = oracle.rel_frobenius(out.cpu().numpy(), int(lg.item()), M, e)
            check_float(err, prec, n, A, M, e, what="served")
    lat = server.latencies_us()
    assert len(lat) == len(reqs) and np.all(lat > 0)
    server.close()
    plan.close()


def test_bad_request_fails_alone():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    server = mpw.Server(64, "fp32", hbm_budget_bytes=8 << 20, max_inflight=4)
    good = wl.modp_uniform(20, 101, 1)
    bad = good.copy()
    bad[3, 3] = 101  # entry >= p
    outs = []
    ts = []
    for A in (good, bad):
        dA = to_dev(A.view(np.int32))
        out = torch.empty_like(dA)
        outs.append((dA, out))
        ts.append(server.submit(dA, 9, out, kind=1, p=101))
    assert server.wait(ts[0]) == mpw.OK
    assert server.wait(ts[1]) == mpw.EINVAL
    want, _ = oracle.matpow_modp(good, 9, 101)
    assert np.array_equal(outs[0][1].cpu().numpy().view(np.uint32).astype(np.uint64), want)
    # a request larger than the whole budget is refused at submission
    big = torch.zeros((64, 64), device="cuda")
    tiny_server = mpw.Server(64, "fp32", hbm_budget_bytes=4096, max_inflight=2)
    with pytest.raises(mpw.MatpowError):
        tiny_server.submit(big, 5, big)
    tiny_server.close()
    server.close()


def test_poll_unknown_ticket_and_eagain():
    from paper_1204_3052_gb300 import matpow as mpw
    server = mpw.Server(64, "fp32", hbm_budget_bytes=8 << 20, max_inflight=4)
    assert server.poll(12345) == mpw.EINVAL
    server.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_tensor_core_modp_requests_and_bad_entry(prec):
    # mod-p requests above N = 64 run on the tensor cores (byte slices) inside
    # the server's grouped levels; one bad entry fails only its own request
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    server = mpw.Server(512, prec, hbm_budget_bytes=64 << 20, max_inflight=8)
    p = 65521
    cases = [(100, 7), (257, 1000), (512, 2 ** 30 - 1), (130, 2)]
    bad = wl.modp_uniform(100, p, 77)
    bad[5, 9] = p
    subs = []
    for i, (N, n) in enumerate(cases):
        A = wl.modp_uniform(N, p, 60 + i)
        dA = to_dev(A.view(np.int32))
        out = torch.empty_like(dA)
        subs.append((A, n, dA, out, server.submit(dA, n, out, kind=1, p=p)))
    dB = to_dev(bad.view(np.int32))
    oB = torch.empty_like(dB)
    tb = server.submit(dB, 33, oB, kind=1, p=p)
    for A, n, dA, out, t in subs:
        assert server.wait(t) == mpw.OK
    assert server.wait(tb) == mpw.EINVAL
    torch.cuda.synchronize()
    for A, n, dA, out, t in subs:
        want, _ = oracle.matpow_modp(A, n, p)
        assert np.array_equal(out.cpu().numpy().view(np.uint32).astype(np.uint64), want), (A.shape[0], n)
    server.close()
