"""GB300-native DysonNet / ABACUS local estimator (arXiv 2603.11189).

The compute path is the CUDA library ``libdysonnet.so`` (sources in csrc/,
C ABI in include/dysonnet.h); ``dysonnet`` is its Python binding.
"""
from . import build  # noqa: F401

__all__ = ["build", "dysonnet"]
