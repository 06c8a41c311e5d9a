"""GB300 tensor-product multigrid for the lat-lon pressure-correction system.

The solver (Sections 2.1-2.3 of the paper) runs as hand-written sm_103a CUDA
kernels in libtpmg.so behind the C ABI of include/tpmg.h; this package is
the thin Python binding over it.  Importing the package does not load the
library; the first handle does, and fails loudly if it has not been built.
"""
from ._lib import (  # noqa: F401
    MG_METHOD_CG,
    MG_METHOD_STATIONARY,
    MG_PREC_FP32,
    MG_PREC_FP64,
    MGError,
    default_params,
    load,
)


def __getattr__(name):
    if name in ("MGHandle", "MGBatch", "MGSolveFn", "mg_solve_fn", "NSHandle", "NSSolveFn",
                "ns_solve_fn", "cast_fp32", "update_fp64"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
