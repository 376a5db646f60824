"""GB300-native GPCG: gradient projection + conjugate gradients for
bound-constrained quadratic programs with stencil Hessians, on hand-written
sm_103a CUDA kernels behind the C ABI of include/gpcg.h.

The Python names mirror the C entry points (see :mod:`.gpcg`)."""
from .gpcg import (CG_EXTRACTED, CG_MASKED, ERR_ARG, ERR_BUDGET, ERR_CANCELLED,  # noqa: F401
                   ERR_CUDA, ERR_INFEASIBLE, ERR_LINESEARCH, ERR_MAXIT, ERR_NUMERIC, ERR_OOM,
                   ERR_PENDING, ERR_TIMEOUT, FP64, MIXED, OK, PATH_AUTO, PATH_ENGINE, PATH_RESIDENT,
                   PRECOND_JACOBI, PRECOND_NONE,
                   PRECOND_TILE, GpcgError, Problem, Server, default_options, gpcg_masked_spmv,
                   gpcg_problem_create, gpcg_problem_update, gpcg_problem_update_async,
                   gpcg_reduced_system, gpcg_result,
                   gpcg_solve, gpcg_solve_batch, gpcg_tile_precondition, gpcg_time_masked_spmv,
                   gpcg_time_masked_spmv_stream,
                   library_path, load)
