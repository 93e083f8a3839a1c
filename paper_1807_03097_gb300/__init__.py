"""GB300-native isogeometric EFIE with interpolation-based FMM (arXiv 1807.03097).

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/efie.h``);
``efie`` is its ctypes binding.
"""
from . import efie  # noqa: F401
from .efie import Solver, options  # noqa: F401
