"""GB300-native integer matrix power A^n (arXiv 1204.3052) behind the libmatpow C-ABI.

``paper_1204_3052_gb300.matpow`` is the Python binding of ``include/matpow.h``;
``paper_1204_3052_gb300.workloads`` draws the seeded synthetic inputs.  Neither
is imported here, so importing the package loads no native code.
"""
__all__ = ["matpow", "workloads"]
