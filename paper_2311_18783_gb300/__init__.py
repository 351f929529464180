"""GB300 (sm_103a) library for the GenEO-type two-level additive Schwarz
preconditioner of positive Maxwell problems (arXiv 2311.18783).

The computation lives in the C-ABI shared library ``libgeneo.so`` (see
``include/geneo.h``); this package only marshals arguments.  Every entry
point loads the library first and raises if it has not been built: there is
no CPU fallback.
"""
from .api import (GeneoError, Mlp, Options, Solver, compose, load_library, shard_problems,
                  PREC_FP64, PREC_FP32, PREC_BF16, COARSE_NONE, COARSE_SNK, COARSE_NK,
                  TAU_RECIPROCAL, TAU_PAPER, PENCIL_FILTERED, PENCIL_CLASSICAL)

__all__ = ["GeneoError", "Mlp", "Options", "Solver", "compose", "load_library", "shard_problems",
           "PREC_FP64", "PREC_FP32", "PREC_BF16", "COARSE_NONE", "COARSE_SNK", "COARSE_NK",
           "TAU_RECIPROCAL", "TAU_PAPER", "PENCIL_FILTERED", "PENCIL_CLASSICAL"]
