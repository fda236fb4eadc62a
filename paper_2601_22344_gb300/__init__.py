"""GB300 (sm_103a) Randomly Pivoted LU.

The product is the CUDA library behind include/rplu.h (built in-tree into
_build/librplu.so by build.py); this package is its Python binding.
Importing it loads the library and raises if it has not been built.
"""
from .binding import (EXPORTED, RPLU_ERR_CUDA, RPLU_ERR_INVALID, RPLU_ERR_NOMEM, RPLU_ERR_TIMEOUT,  # noqa: F401
                      RPLU_NOT_CONVERGED, RPLU_OK, Job, Opts, Result, RPLUError, lib, rplu_cauchy, rplu_dense,
                      status_string, version)
