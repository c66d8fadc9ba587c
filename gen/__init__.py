"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

This package only *generates data*. It holds none of the method's arithmetic (no
Gram-Schmidt, no projection, no error indicator), so the oracle and the CUDA path can both
consume it without sharing any code of the method.
"""
from .inputs import (  # noqa: F401
    haar_orthonormal,
    lowrank_haar,
    decay_matrix_c1,
    image_like_factors,
    image_like_u8,
    u8_to_unit_f64,
    parametric_params,
    parametric_snapshots,
    parametric_snapshots_torch,
    paper_rank_function,
    paper_approx_function,
    orthogonal_columns,
    row_weights,
    out_of_sample,
    batch_specs,
    decay_spectrum,
    lowrank_torch,
)
