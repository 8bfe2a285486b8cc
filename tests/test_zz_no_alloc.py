"""The no-allocation residual entry point (jac_residual_dense_noalloc).

Some callers cannot allocate device memory where they need a residual (a
framework step that forbids allocation, a locked memory pool, a callback
that must not block on the allocator). This entry point takes the caller's
dense device grid and keeps its scratch in a fixed static device array.
Here it is called through the C ABI and checked against the context-based
jac_residual on the same grid, within the residual tolerance the other
tests use (1e-12 relative), on two calls in a row. This file is collected
last so that a run stopping at the first failure has run every other test.
"""

import numpy as np
import pytest

import synth
from paper_2202_11819_gb300 import Jacobi3D, _lib

pytestmark = pytest.mark.gpu

BC = (1.0, 0.25, 0.0, 0.5, 0.125, 0.75)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def context_residual(u, block):
    nz, ny, nx = u.shape
    dtype = "f32" if u.dtype == np.float32 else "f64"
    with Jacobi3D((nx, ny, nz), block, dtype=dtype, bc=BC) as J:
        J.write(u)
        return J.residual()


def noalloc_residual(torch, u):
    nz, ny, nx = u.shape
    dev = torch.from_numpy(np.ascontiguousarray(u).reshape(-1)).to("cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    dt = _lib.JAC_F32 if u.dtype == np.float32 else _lib.JAC_F64
    s = torch.cuda.current_stream()
    _lib.jac_residual_dense_noalloc(dev.data_ptr(), dt, nx, ny, nz, BC, out.data_ptr(), s.cuda_stream)
    s.synchronize()
    return out.item()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_noalloc_residual_matches_context_residual_twice(torch_cuda, dtype):
    # first call: a larger grid; second call: a smaller one, so the second
    # reads only slots it wrote itself although the array keeps the first
    # call's contents
    u1 = synth.grid_uniform01(31, 70, 45, 33).astype(dtype)
    u2 = synth.grid_uniform01(32, 20, 9, 14).astype(dtype)
    for u, block in ((u1, (32, 16, 11)), (u2, (8, 9, 7))):
        want = context_residual(u, block)
        got = noalloc_residual(torch_cuda, u)
        assert abs(got - want) <= 1e-12 * want


def test_noalloc_rejects_grids_beyond_the_scratch(torch_cuda):
    dev = torch_cuda.zeros(1, dtype=torch_cuda.float64, device="cuda")
    out = torch_cuda.zeros(1, dtype=torch_cuda.float64, device="cuda")
    # ceil(nx/32) * ceil(ny/8) = 4096 * 32 > 65536 partial slots
    with pytest.raises(_lib.JacError) as e:
        _lib.jac_residual_dense_noalloc(dev.data_ptr(), _lib.JAC_F64, 32 * 4096, 8 * 32, 1, BC, out.data_ptr())
    assert e.value.code == _lib.JAC_EINVAL
