"""CPU oracle for the tournament-pivoting LU hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``lu_oracle.c`` (plain FP64
C, built with gcc) through ctypes and shares nothing with the GPU library.

Parity status of each function (what pins it is in ``tests/test_oracle_*.py``):

* ``lu_factor``      -- pinned: GEPP special cases against LAPACK getrf,
  closed-form L*U products, permutation and triangular matrices, cofactor
  determinants, invariants, loop-bound counts of Section 6, and an independent
  exact-rational tournament on tiny inputs.
* ``tslu_select``    -- pinned through the same tests (b = 1 and one-leaf
  cases reduce to partial pivoting; brute force on tiny inputs).
* ``lu_solve``       -- pinned against numpy.linalg.solve and exact integer
  systems.
* ``backward_error`` -- pinned against closed forms (exact solutions give 0,
  hand-computed small cases).
* ``lu_factor_f32`` / ``lu_solve_f32`` -- the same code instantiated for
  binary32; pinned by LAPACK sgetrf (b = 1) and exact dyadic L*U products.
* ``round_lowp``     -- pinned against torch's bfloat16 / float8_e4m3fn
  conversions (round to nearest even) and hand-worked ties and saturation.
* ``chol_factor`` / ``chol_solve`` (binary64 and binary32) -- pinned by exact
  integer factors L (A = L L^T recovered bit for bit), numpy's Cholesky and
  solve, the info of matrices with a known first non-positive pivot, the
  untouched upper triangle, and the 1 x 1 and diagonal special cases.
* ``e4m3_exponent``, ``gemm_lowp`` -- pinned by hand-worked exponents and by
  exactly representable operands, where the update equals the binary64
  product.
"""
from .oracle import (  # noqa: F401
    build,
    lib_path,
    lu_factor,
    lu_solve,
    tslu_select,
    backward_error,
    set_threads,
    lu_factor_f32,
    lu_solve_f32,
    round_lowp,
    e4m3_exponent,
    gemm_lowp,
    chol_factor,
    chol_solve,
)
