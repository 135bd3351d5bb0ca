"""Seeded synthetic inputs for MSP: dense PSD matrices A, right-hand sides b.

This package holds input generators only. It contains none of the method's
arithmetic (no sketching, no preconditioner, no solver), so both the CUDA path
and the FP64 oracle can draw identical inputs from it without sharing any code
of the method itself.
"""

from .generators import (  # noqa: F401
    outlier_spectrum,
    householder_spectrum,
    spectrum_matrix,
    gaussian_square,
    householder_matrix,
    householder_factors,
    householder_lowrank,
    rbf_points,
    rbf_kernel,
    rhs,
    Workload,
    make_workload,
    WORKLOADS,
    BatchSpec,
    batch_specs,
    batch_instance,
    svd_matrix,
    tall_matrix,
)
