"""Workload recipes: boundary values, batch instance shapes, serving trace.

Every draw comes from SplitMix64 (``synth.splitmix``) so the same seed gives
the same workload on every machine. None of this is Jacobi arithmetic.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .splitmix import uniform01

# Dirichlet values of the six ghost planes, in the order -x, +x, -y, +y, -z, +z:
# 1.0 outside the x = 0 face, 0.0 outside the other five faces.
DIRICHLET_X0 = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)

# Per-axis sizes of the batched workload: 32, 48, ..., 192 (11 values).
BATCH_AXIS_VALUES = tuple(range(32, 193, 16))


def batch_instance_dims(n_instances: int, seed: int = 0) -> list[tuple[int, int, int]]:
    """Shape (nx, ny, nz) of each instance of the batched workload: every axis
    drawn independently and uniformly from 32, 48, ..., 192. Instance ``i``
    uses outputs 3i, 3i+1, 3i+2 of the stream at ``seed``."""
    u = uniform01(seed, 0, 3 * n_instances).reshape(n_instances, 3)
    k = np.minimum((u * len(BATCH_AXIS_VALUES)).astype(np.int64), len(BATCH_AXIS_VALUES) - 1)
    vals = np.asarray(BATCH_AXIS_VALUES)[k]
    return [tuple(int(v) for v in row) for row in vals]


@dataclass(frozen=True)
class SolveRequest:
    """One request of the serving trace."""

    rid: int
    arrival_s: float
    dims: tuple[int, int, int]
    dtype: str  # "f64" or "f32"
    seed: int  # seed of the request's initial interior


def serving_trace(n_requests: int = 2000, rate_per_s: float = 200.0, seed: int = 0,
                  lo: int = 32, hi: int = 384) -> list[SolveRequest]:
    """Poisson arrivals (exponential gaps, mean 1/rate), each axis log-uniform in
    [lo, hi] and rounded, dtype f32 or f64 with probability 1/2 each. Request
    ``r`` uses stream outputs 5r .. 5r+4 (gap, three axes, dtype) and its
    interior is drawn with seed ``seed * 1_000_003 + r + 1``."""
    u = uniform01(seed, 0, 5 * n_requests).reshape(n_requests, 5)
    t = 0.0
    out = []
    la, lb = math.log(lo), math.log(hi)
    for r in range(n_requests):
        t += -math.log1p(-float(u[r, 0])) / rate_per_s
        dims = tuple(int(min(hi, max(lo, round(math.exp(la + float(u[r, q]) * (lb - la)))))) for q in (1, 2, 3))
        dtype = "f32" if float(u[r, 4]) < 0.5 else "f64"
        out.append(SolveRequest(r, t, dims, dtype, seed * 1_000_003 + r + 1))
    return out
