"""Shared test helpers: tolerances and device plumbing (no method arithmetic)."""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "matpow.h")


def header_functions():
    """Names of the functions include/matpow.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(matpow_[a-z0-9_]+)\s*\(", text)))


def float_tol(n: int) -> float:
    """rel. Frobenius bound for float32-class results: 2e-5 * ceil(log2 n).

    n = 1 is a copy and must be exact (bound 1e-7); n = 0 the identity.
    """
    if n <= 1:
        return 1e-7
    return 2e-5 * math.ceil(math.log2(n))


def gate(n: int, floor_rel: float) -> float:
    """max(2e-5*ceil(log2 n), 2 x the error of a float32 run of the same method)."""
    return max(float_tol(n), 2.0 * floor_rel)


def to_dev(a, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)
