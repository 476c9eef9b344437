"""FP32 SIMT products on 64- and 128-wide tiles (GPU).  A launch takes 64 x 64
tiles when its 128 x 128 tiles would not fill the SMs; every element is summed
in the same k order on either, so the two must agree bit for bit.  One
N = 1024 power alone runs on 64-wide tiles (64 tiles of 128 < 152 SMs), the
same power in a batch of three on 128-wide ones (192 tiles of 128)."""
import numpy as np
import pytest

import oracle
from helpers import to_dev
from paper_1204_3052_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_64_and_128_wide_tiles_agree_bitwise():
    import torch
    from paper_1204_3052_gb300 import matpow as mpw
    N = 1024
    As = [wl.gaussian(N, s) for s in (11, 12, 13)]
    plan = mpw.Plan(N, "fp32")
    for n in (2, 3, 6):
        alone, la = plan.f32(to_dev(As[0]), n, mantissa=True)
        plan.check()
        outs = [torch.empty((N, N), dtype=torch.float32, device="cuda") for _ in As]
        lg = torch.zeros(len(As), dtype=torch.int64, device="cuda")
        mpw._check(mpw.matpow_batched(plan.h, [to_dev(a) for a in As], [N] * 3, [n] * 3, outs, lg), plan.h)
        plan.check()
        assert int(la.item()) == int(lg[0].item()), n
        assert torch.equal(alone, outs[0]), (n, (alone - outs[0]).abs().max().item())
    plan.close()


def test_128_wide_tiles_against_oracle_rows():
    # N = 2048 alone: 256 tiles of 128 >= the SMs, so 128-wide tiles; rows of
    # A^2 by the float64 oracle, rows of A^3 as those rows times A in float64
    from paper_1204_3052_gb300 import matpow as mpw
    N = 2048
    A = wl.gaussian(N, 21)
    plan = mpw.Plan(N, "fp32")
    ranges = [(0, 8), (1020, 1030), (N - 6, N)]
    A2 = {r: oracle.gemm_rows_f64(A, A, *r) for r in ranges}
    for n in (2, 3):
        got, lg = plan.f32(to_dev(A), n, mantissa=True)
        plan.check()
        G = got.cpu().numpy()
        for r0, r1 in ranges:
            want = A2[(r0, r1)] if n == 2 else A2[(r0, r1)] @ A.astype(np.float64)
            rows = np.ldexp(G[r0:r1].astype(np.float64), int(lg.item()))
            rel = np.linalg.norm(rows - want) / np.linalg.norm(want)
            assert rel <= 2e-5 * int(np.ceil(np.log2(n))), (n, r0, rel)
    plan.close()
