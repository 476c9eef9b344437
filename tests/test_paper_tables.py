"""The paper's own workloads (Sec. 5.2 tables, transcribed in tests/golden/).

The tables give no matrix values, so they pin only the structure of the
method: every power the paper runs is 2^k, which the square-and-multiply
schedule covers with k products, against n-1 for the naive method (Sec. 4.2).
"""
import math
import os

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def rows():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            N, n, naive, cpu, ours, ratio = line.split()
            out.append((int(N), int(n), float(naive), float(cpu), float(ours), float(ratio)))
    return out


def test_table_has_all_sizes_and_powers():
    r = rows()
    assert {N for N, *_ in r} == {64, 128, 256, 512}
    assert len(r) == 16


def test_paper_powers_take_log2_products():
    for N, n, *_ in rows():
        k = int(math.log2(n))
        assert 2 ** k == n
        assert oracle.gemm_count(n) == k          # "log(N)" products, Sec. 4.3
        assert len(oracle.schedule(n)) == k + 1   # levels 0..k, bit k copies


def test_ratio_column_consistent_with_rounded_times():
    # ours_vs_naive = naive / ours up to the 0.01 s rounding of both times
    for N, n, naive, cpu, ours, ratio in rows():
        lo = max(naive - 0.005, 0.0) / (ours + 0.005)
        hi = (naive + 0.005) / max(ours - 0.005, 1e-9)
        assert lo * 0.99 <= ratio <= hi * 1.01, (N, n)
