"""GB300-native steady shallow-water Newton multigrid (arXiv 2505.10857).

The compute path is the CUDA library ``libnswe_gb300.so`` (C ABI declared in
``include/nswe.h``), bound by :mod:`paper_2505_10857_gb300.nswe`. Importing
this package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
__all__ = ["inputs", "nswe", "build"]
