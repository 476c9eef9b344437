"""Every choice in the tuned tile table passes parity (GPU).

For each rule of the shipped table (and a few hand-written rules that force
each launch shape), powers of orders at both ends of the rule's range run on
a plan that carries the table and are checked against the float64 oracle:
whole results up to N = 1024, sampled rows of A^2 recomputed in float64
above.  Batches with orders in the ranges whose `persist` the table sets are
checked the same way through matpow_batched."""
import os

import numpy as np
import pytest

import oracle
from helpers import check_float, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PREC_NAME = {2: "bf16x3", 3: "bf16x6"}


def _table():
    from paper_1204_3052_gb300 import matpow as mpw
    if not os.path.exists(mpw.DEFAULT_TILE_TABLE):
        pytest.skip("no tuned table shipped")
    st, rules = mpw.matpow_tile_table_parse(open(mpw.DEFAULT_TILE_TABLE).read())
    assert st == mpw.OK
    return rules


def _check_power(plan, prec, N, n, seed):
    A = wl.gaussian(N, seed)
    dA = to_dev(A)
    out, lg = plan.f32(dA, n, mantissa=True)
    plan.check()
    if N <= 1024:
        M, e, _ = oracle.matpow_f64(A, n)
        err = oracle.rel_frobenius(out.cpu().numpy(), int(lg.item()), M, e)
        check_float(err, prec, n, A, M, e, what="tile table")
        return
    # large orders: A^2 on sampled rows, each row a float64 vector-matrix product
    assert n == 2
    got = np.ldexp(out.cpu().numpy().astype(np.float64), int(lg.item()))
    A64 = A.astype(np.float64)
    rows = np.random.default_rng(seed).choice(N, 8, replace=False)
    want = A64[rows] @ A64
    err = float(np.linalg.norm(got[rows] - want) / np.linalg.norm(want))
    assert err <= (2e-5 if prec == "bf16x6" else 2e-3), (prec, N, err)


def _orders(rule):
    lo, hi = rule["n_lo"], rule["n_hi"]
    return sorted({max(lo + 1, 65), hi}) if hi > 64 else []


def test_every_tabled_single_power_choice_matches_oracle():
    from paper_1204_3052_gb300 import matpow as mpw
    rules = _table()
    plans = {}
    for r in rules:
        prec = PREC_NAME.get(r["precision"])
        if prec is None:
            continue
        for N in _orders(r):
            if N > 8192:
                continue
            key = (prec, N > 1024)
            if key not in plans:
                plans[key] = mpw.Plan(8192 if N > 1024 else 1024, prec, tile_table=mpw.DEFAULT_TILE_TABLE)
            _check_power(plans[key], prec, N, 2 if N > 1024 else 77, N)
    for p in plans.values():
        p.close()


def test_every_tabled_batched_choice_matches_oracle():
    from paper_1204_3052_gb300 import matpow as mpw
    rules = [r for r in _table() if r["persist"] >= 0 and r["n_hi"] <= 1024]
    for prec in ("bf16x3", "bf16x6"):
        mine = [r for r in rules if PREC_NAME.get(r["precision"]) == prec]
        if not mine:
            continue
        Ns = [N for r in mine for N in _orders(r)]
        ns = [77, 2, 13, 1000][:len(Ns)] * (len(Ns) // 4 + 1)
        ns = ns[:len(Ns)]
        As = [wl.gaussian(N, 500 + i) for i, N in enumerate(Ns)]
        plan = mpw.Plan(max(Ns), prec, tile_table=mpw.DEFAULT_TILE_TABLE)
        import torch
        lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
        outs = plan.batched([to_dev(a) for a in As], ns, log2=lg)
        plan.check()
        for i, (A, n) in enumerate(zip(As, ns)):
            M, e, _ = oracle.matpow_f64(A, n)
            err = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lg[i].item()), M, e)
            check_float(err, prec, n, A, M, e, what="tile table batch")
        plan.close()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_forced_shapes_match_oracle(prec):
    # each launch shape the table can name, forced on one range of orders
    from paper_1204_3052_gb300 import matpow as mpw
    shapes = [{"chain": 1, "bn": 64, "split_k": 1}, {"chain": 1, "bn": 64, "split_k": 2},
              {"chain": 0, "bn": 64}]
    if prec == "bf16x3":
        shapes += [{"chain": 1, "bn": 64, "split_k": 4}, {"chain": 1, "bn": 128}, {"chain": 0, "bn": 128}]
    plan = mpw.Plan(1024, prec)
    for sh in shapes:
        rule = dict({"precision": prec, "n_lo": 64, "n_hi": 1024, "persist": -1, "split_k": -1}, **sh)
        plan.set_tile_table([rule])
        for N in (65, 300, 700):
            _check_power(plan, prec, N, 77, N + 3)
    # batched: persistent and per-tile levels, 64-column tiles
    import torch
    As = [wl.gaussian(N, 7 * N) for N in (80, 200, 256)]
    for persist in (1, 0):
        plan.set_tile_table([{"precision": prec, "n_lo": 64, "n_hi": 1024, "persist": persist, "bn": 64}])
        lg = torch.zeros(3, dtype=torch.int64, device="cuda")
        outs = plan.batched([to_dev(a) for a in As], [5, 300, 17], log2=lg)
        plan.check()
        for i, (A, n) in enumerate(zip(As, [5, 300, 17])):
            M, e, _ = oracle.matpow_f64(A, n)
            err = oracle.rel_frobenius(outs[i].cpu().numpy(), int(lg[i].item()), M, e)
            check_float(err, prec, n, A, M, e, what="persist=%d" % persist)
    plan.close()
