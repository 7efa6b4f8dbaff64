"""GB300 SELL-C-sigma augmented SpMMV (GHOST, arxiv 1507.08101).

The compute path is the CUDA library built from ``csrc/`` (see
``include/sellcs.h``); this package holds its build step and a thin ctypes
binding.  Importing the package does not load the library; the first call
does, and fails loudly if it has not been built.
"""
from .sellcs import (SellMatrix, SpError, spmv, spmv_adjoint, lib, library_path,  # noqa: F401
                     sp_device_sm_count)
