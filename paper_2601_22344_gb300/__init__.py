"""GB300 (sm_103a) Randomly Pivoted LU.

The product is the CUDA library behind include/rplu.h (built in-tree into
_build/librplu.so by build.py); this package is its Python binding.  The
library is loaded on first use of any binding attribute (rplu_dense, ...);
that raises ImportError if it has not been built.  `paper_2601_22344_gb300.build`
can be imported without it.
"""
import importlib

_BINDING_NAMES = {"EXPORTED", "RPLU_ERR_CUDA", "RPLU_ERR_INVALID", "RPLU_ERR_NOMEM", "RPLU_ERR_TIMEOUT",
                  "RPLU_NOT_CONVERGED", "RPLU_CANCELLED", "RPLU_OK", "Job", "Opts", "Result", "RPLUError", "lib",
                  "rplu_bh_bounds", "rplu_bh_plan_stats", "rplu_cur_aaa", "rplu_barycentric", "CurAaa", "rplu_cauchy", "rplu_cauchy_cur", "rplu_toeplitz3_cur", "rplu_sparse_cur", "rplu_cauchy_like", "rplu_dense",
                  "status_string", "version"}


def __getattr__(name):
    if name in ("binding", "batch", "build", "serve"):
        return importlib.import_module("." + name, __name__)
    if name in _BINDING_NAMES:
        return getattr(importlib.import_module(".binding", __name__), name)
    raise AttributeError(name)
