"""The C-ABI library builds, loads and exports every declared symbol (CPU only).

No compute call is made here: this container has no GPU.
"""
import ctypes
import subprocess

import pytest

from helpers import header_functions
from paper_1204_3052_gb300 import matpow as mpw


@pytest.fixture(scope="module")
def lib():
    return mpw.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("matpow_plan", "matpow_f32", "matpow_batched", "matpow_mod_p",
                     "matpow_submit", "matpow_poll", "matpow_sync", "matpow_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", mpw.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing
    for n in header_functions():
        assert hasattr(lib, n)


def test_binding_names_match_header():
    assert sorted(mpw.EXPORTS) == header_functions()


def test_gemm_count_host_only(lib):
    import oracle
    for n in (0, 1, 2, 3, 7, 100, 1024, 2 ** 20, 2 ** 30 - 1, 2 ** 63 + 5):
        want = oracle.gemm_count(n) if n < 2 ** 40 else ((n.bit_length() - 1) + bin(n).count("1") - 1)
        assert mpw.matpow_gemm_count(n) == want


def test_workspace_size_grows_with_n(lib):
    a = mpw.matpow_workspace_size(512, "bf16x3")
    b = mpw.matpow_workspace_size(1024, "bf16x3")
    assert 0 < a < b
    assert mpw.matpow_workspace_size(0, "fp32") == 0


def test_plan_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.matpow_plan(ctypes.byref(h), 64, 0, 0, 0)
    assert st in (mpw.ECUDA, mpw.EINVAL)
    assert h.value is None
    assert lib.matpow_last_error(None)


def test_null_plan_rejected(lib):
    assert lib.matpow_f32(None, None, 4, 2, None, None, None) == mpw.EINVAL
    assert lib.matpow_mod_p(None, None, 4, 2, 7, None, None) == mpw.EINVAL
    assert lib.matpow_sync(None, None) == mpw.EINVAL
    assert lib.matpow_plan_destroy(None) == mpw.OK
