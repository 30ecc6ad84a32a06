"""GB300-native shifted-HSS Helmholtz solver (arXiv 2506.18694, hot path).

``hh`` is the ctypes binding of the C ABI in ``include/hh.h``; ``inputs`` draws the
seeded synthetic workloads.  Importing the package loads nothing; the CUDA library
is loaded on first use and its absence is an error, never a fallback.
"""

__all__ = ["hh", "inputs"]
