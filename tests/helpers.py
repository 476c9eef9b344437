"""Shared test helpers: tolerances and device plumbing (no method arithmetic).

Float bounds.  The stated bound for a float32-class result of A^n is the
relative Frobenius error 2e-5 ceil(log2 n) (1e-7 for n = 1, an exact copy).
Where a test's input makes that bound out of reach for any float32-class
arithmetic (Gaussian inputs at large n: the error of the dominant eigenvalues
doubles with each squaring), the bound takes the larger of the stated one and
a floor that depends on the path's class:

* float32-class paths (FP32 SIMT, and BF16X6, whose three exact slices keep
  24 bits per block): 8 x the deviation of the float64 chain whose stored
  products carry normwise perturbations of 2^-24 (``oracle.perturbed_sqmul``,
  two seeds): how far storage errors of a float32-class format carry through
  this input's chain.  No model of the kernels' own arithmetic enters it.
* lower-precision paths (plain BF16 and BF16X3, 8 and 16 bits): 2 x the
  error of the path's operand rounding emulated on the CPU
  (``oracle.emu_sqmul``, pinned in tests/test_oracle_yardsticks.py).

Orders N <= 64 run the float32 on-chip chain whatever the precision, so they
take the float32-class bound.  ``check_float`` prints which term bound.
"""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "matpow.h")

FLOAT32_CLASS = ("fp32", "bf16x6")
EMU = {"bf16": "bf16", "bf16x3": "bf16x3blk"}
PERTURBATION = 2.0 ** -24
PERTURBATION_FACTOR = 8.0


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


def float32_class_floor(A, n, M, e) -> float:
    """Deviation of the float64 chain with 2^-24 normwise storage perturbations."""
    import oracle
    return max(oracle.rel_frobenius(*oracle.perturbed_sqmul(A, n, PERTURBATION, seed), M, e)
               for seed in (0, 1))


def float_bound(prec, n, A, M, e, stated_only=False, tiny_max=64):
    """(bound, term) for a float result of A^n (oracle M 2^e) on path `prec`."""
    t = float_tol(n)
    if stated_only or n <= 1:
        return t, "stated"
    if prec in FLOAT32_CLASS or A.shape[0] <= tiny_max:
        f = PERTURBATION_FACTOR * float32_class_floor(A, n, M, e)
        return (t, "stated") if t >= f else (f, "float32-class floor (8 x 2^-24 perturbation)")
    import oracle
    Me, ee = oracle.emu_sqmul(A, n, EMU[prec])
    f = 2.0 * oracle.rel_frobenius(Me, ee, M, e)
    return (t, "stated") if t >= f else (f, "2 x emulated %s" % EMU[prec])


def check_float(err, prec, n, A, M, e, stated_only=False, tiny_max=64, what=""):
    """Assert err within float_bound and print which term bound."""
    b, term = float_bound(prec, n, A, M, e, stated_only, tiny_max)
    print("%s prec=%s N=%d n=%d rel_F=%.3e bound=%.3e [%s]" % (what, prec, A.shape[0], n, err, b, term))
    assert err <= b, (what, prec, A.shape[0], n, err, b, term)


def to_dev(a, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)
