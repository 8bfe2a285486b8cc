"""Seeded synthetic inputs for Jacobi3D runs.

This package is shared by the oracle-side tests and the CUDA-side tests and
benchmark. It holds no part of the Jacobi method's arithmetic: it only draws
the initial interior values, the boundary values and the workload shapes that
both sides are then given as inputs.
"""

from .splitmix import splitmix64, uniform01, grid_uniform01, grid_uniform01_f32
from .workloads import (
    DIRICHLET_X0,
    batch_instance_dims,
    serving_trace,
)

__all__ = [
    "splitmix64",
    "uniform01",
    "grid_uniform01",
    "grid_uniform01_f32",
    "DIRICHLET_X0",
    "batch_instance_dims",
    "serving_trace",
]
