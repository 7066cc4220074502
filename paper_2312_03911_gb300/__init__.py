"""GB300-native gradient-guided nested sampling (arXiv 2312.03911).

The compute path is the CUDA library ``libggns.so`` (sm_103a) behind the C ABI in
``include/ggns.h``; :mod:`paper_2312_03911_gb300.ggns` is its thin ctypes binding.
Importing this package loads nothing; the binding loads the library on first use
and raises if it is missing (there is no CPU fallback).
"""
__all__ = ["ggns", "workloads"]
