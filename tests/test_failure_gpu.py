"""The timeout path of the bounded waits, without a GPU fault: one CTA waits
on an mbarrier that nothing arrives at, gives up after a short budget and
records the timeout; the host reads MATPOW_ETIMEDOUT from matpow_sync and the
plan keeps working."""
import time

import numpy as np
import pytest

import oracle
from helpers import check_float, to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports_timeout():
    from paper_1204_3052_gb300 import matpow as mpw
    plan = mpw.Plan(128, "bf16x6")
    t0 = time.perf_counter()
    assert mpw.matpow_selftest_wait_timeout(plan.h, 20_000_000) == mpw.OK  # 20 ms of GPU time
    st = plan.sync()
    elapsed = time.perf_counter() - t0
    assert st == mpw.ETIMEDOUT
    assert 0.02 <= elapsed < 10.0
    assert "wait" in mpw.load().matpow_last_error(plan.h).decode()
    # the status word was cleared and the plan still computes
    A = wl.gaussian(100, 3)
    out, lg = plan.f32(to_dev(A), 9, mantissa=True)
    assert plan.sync() == mpw.OK
    M, e, _ = oracle.matpow_f64(A, 9)
    err = oracle.rel_frobenius(out.cpu().numpy().astype(np.float64), int(lg.item()), M, e)
    check_float(err, "bf16x6", 9, A, M, e, stated_only=True, what="after the timeout")
    plan.close()


def test_selftest_rejects_budget_out_of_range():
    from paper_1204_3052_gb300 import matpow as mpw
    plan = mpw.Plan(64, "fp32")
    assert mpw.matpow_selftest_wait_timeout(plan.h, 10) == mpw.EINVAL
    assert mpw.matpow_selftest_wait_timeout(plan.h, 10 ** 11) == mpw.EINVAL
    assert plan.sync() == mpw.OK
    plan.close()
