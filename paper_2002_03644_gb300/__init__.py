"""GB300 (sm_103a) hybrid lattice Boltzmann step of Renard, Feng, Boussuge and
Sagaut (arXiv 2002.03644).

Submodules:
  hlbm    -- ctypes binding of libhlbm (include/hlbm.h), the CUDA library
  inputs  -- seeded synthetic initial fields and case parameters
  build   -- nvcc build of libhlbm.so for sm_103a

Importing the package loads nothing; the library is opened on first use.
"""

__all__ = ["hlbm", "inputs", "build"]
