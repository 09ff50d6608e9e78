"""GB300-native relativistic SHASTA solver (arXiv:1206.0919).

The solver is the CUDA library ``libshasta.so`` behind the C ABI of
``include/shasta.h``; ``paper_1206_0919_gb300.shasta`` is its ctypes binding
and ``paper_1206_0919_gb300.workloads`` draws seeded initial data.
Importing the package loads nothing; the binding loads the library on first
use and raises if it has not been built.
"""
__all__ = ["shasta", "workloads", "build"]
__version__ = "0.1.0"
