"""GB300-native pseudoinverse-preconditioned CG for the FD Poisson problem.

The compute path is libtpcg.so (CUDA, sm_103a) behind the C ABI of
include/tpcg.h; this package holds its sources (csrc/), the build script and
a ctypes binding with the same function names.
"""
from .binding import (  # noqa: F401
    BC, PREC, TPCG_FP64, TPCG_MIXED_BF16, TPCG_MIXED_FP16, TPCG_MIXED_TF32, TPCG_OK, TPCG_ZERO_GUESS, Plan, Server,
    TpcgError, lib,
    tpcg_apply_laplacian, tpcg_plan_create, tpcg_plan_destroy, tpcg_plan_device_bytes, tpcg_plan_eigenpairs,
    tpcg_plan_set_stream, tpcg_precond_apply, tpcg_rhs_add_bc, tpcg_solve, tpcg_solve_host, tpcg_strerror,
)
