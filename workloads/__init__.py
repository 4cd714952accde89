"""Seeded synthetic inputs shared by the oracle-side tests and the GPU-side
tests and benchmark.  Nothing here performs any step of the LU or Cholesky method."""
from .generators import (  # noqa: F401
    splitmix64,
    uniform01,
    uniform_pm1,
    normal,
    matrix_uniform,
    matrix_normal,
    matrix_spd,
    householder_diag,
    householder_apply_inverse,
    batch_sizes,
    poisson_arrivals,
)
