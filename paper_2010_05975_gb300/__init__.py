"""GB300-native tournament-pivoting LU (the hot path of COnfLUX,
arXiv:2010.05975) behind a C ABI.

This module is argument marshalling only: every step runs in the CUDA
library built from ``csrc/`` (see ``build.py``).  Importing it does not need
a GPU; calling a compute entry point does, and fails loudly when the library
is missing.  Matrices are row-major torch tensors on a CUDA device.
"""
from ._native import (  # noqa: F401
    LU_ELAUNCH,
    LU_ENOMEM,
    LU_ETIMEOUT,
    LU_EBUSY,
    LU_EUNSUPPORTED,
    LU_ENOTFOUND,
    LU_PREC_F64,
    LU_PREC_F32,
    LU_PREC_BF16,
    LU_PREC_FP8,
    LU_WAIT_SITE_TC,
    LU_WAIT_SITE_SOLVE,
    LuError,
    library,
    library_path,
    exported_symbols,
)
from .serving import Server  # noqa: F401
from .api import (  # noqa: F401
    lu_factor,
    lu_factor_ex,
    lu_solve,
    lu_factor_host,
    lu_factor_f32,
    lu_solve_f32,
    chol_factor,
    chol_solve,
    lu_gemm_lowp,
    lu_residual,
    ir_solve,
    lu_factor_batched,
    lu_solve_batched,
    batched_panel_width,
    set_batched_panel_widths,
    BatchedFactorSolve,
    prof_begin,
    prof_end,
    kernel_launch_count,
    set_wait_config,
)
