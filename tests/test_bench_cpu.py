"""Host-side arithmetic of bench.py (CPU only): the stated tolerance, the
product count and the per-level roofline bound of a batch."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6704.5, "bf16_tflops": 1911.3}


def test_stated_tolerance_and_gemm_count():
    assert bench.stated_tolerance(1) == 1e-7
    assert bench.stated_tolerance(2) == pytest.approx(2e-5)
    assert bench.stated_tolerance(1000) == pytest.approx(2e-4)
    assert [bench.gemm_count(n) for n in (0, 1, 2, 3, 100, 1024)] == [0, 0, 1, 2, 8, 10]


def test_batch_roofline_one_square():
    # N = 128, n = 2: one squaring; three slices read once and written once
    by = 2 * 3 * 128 * 128 * 2.0
    fl = 6 * 2 * 128 ** 3
    want = max(by / 6704.5e9, fl / 1911.3e12) * 1e3
    assert bench.batch_roofline_ms([128], [2], "bf16x6", PEAKS) == pytest.approx(want)


def test_batch_roofline_levels_add_and_group():
    # n = 3: level 0 squares, level 1 multiplies R P (two operands read);
    # two such matrices share each level (the maxima add per level)
    N = 256
    sq = max(2 * 2 * N * N * 2.0 / 6704.5e9, 3 * 2 * N ** 3 / 1911.3e12)
    mul = max(2 * 2 * N * N * 3.0 / 6704.5e9, 3 * 2 * N ** 3 / 1911.3e12)
    assert bench.batch_roofline_ms([N], [3], "bf16x3", PEAKS) == pytest.approx((sq + mul) * 1e3)
    two = bench.batch_roofline_ms([N, N], [3, 3], "bf16x3", PEAKS)
    assert two == pytest.approx((max(2 * 2 * 2 * N * N * 2.0 / 6704.5e9, 2 * 3 * 2 * N ** 3 / 1911.3e12)
                                 + max(2 * 2 * 2 * N * N * 3.0 / 6704.5e9, 2 * 3 * 2 * N ** 3 / 1911.3e12)) * 1e3)
    # orders <= 64 run on chip and n <= 1 has no product
    assert bench.batch_roofline_ms([64, 300], [100, 1], "bf16x6", PEAKS) == 0.0
