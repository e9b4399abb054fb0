"""GB300-native population-annealing engine (arXiv:2207.05535).

The hot path is CUDA in ``csrc/`` compiled to ``_build/libpa.so`` and exposed
through the C ABI of ``include/pa.h``; ``_lib`` mirrors that ABI for Python.
Importing this package loads nothing; ``_lib.load()`` raises when the library
has not been built.
"""
__all__ = ["workloads", "build", "_lib"]
