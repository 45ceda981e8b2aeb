"""Mapping-driven record layouts on GB300 (arXiv 2302.08251, LLAMA).

The compute path is the CUDA library ``libllgb.so`` behind the C ABI declared
in ``include/llgb.h``; :mod:`paper_2302_08251_gb300.llgb` is its thin ctypes
binding.  Importing this package loads nothing native; the binding loads the
library on first use and raises if it is missing.
"""
