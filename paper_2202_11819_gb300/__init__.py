"""GB300-native Jacobi3D: the overdecomposed 7-point Jacobi iteration with
per-iteration halo pack / exchange / unpack of "Improving Scalability with
GPU-Aware Asynchronous Tasks" (Choi, Richards, Kale), all blocks resident in
one GPU's HBM.

The compute path is libjacobi3d.so (hand-written sm_103a CUDA kernels behind
the C ABI of include/jacobi3d.h). This package only marshals arguments
(``_lib``, same names as the C ABI) and offers a small convenience class
(``Jacobi3D``) that uses PyTorch for device memory and streams.
"""

from ._lib import (  # noqa: F401
    JAC_ARITH_EXACT,
    JAC_ARITH_SEQ,
    JAC_F32,
    JAC_F64,
    JAC_MODE_FUSED,
    JAC_MODE_GRAPH,
    JAC_MODE_GRAPH_FUSED,
    JAC_MODE_PERSISTENT,
    JAC_MODE_UNFUSED,
    JacError,
    MODES,
    load,
)
from .solver import Jacobi3D, Jacobi3DBatch, use_torch_allocator  # noqa: F401
