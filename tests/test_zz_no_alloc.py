"""The no-allocation residual entry point (jac_residual_dense_noalloc).

Some callers cannot allocate device memory at the point where they need a
residual: a framework step that forbids allocation, code that runs while a
memory pool is locked, a callback that must not block on the allocator. This
entry point takes the caller's dense device grid and keeps its scratch in a
fixed static device array of the library.

Here it is called through the C ABI on two calls in a row and checked
against the context-based jac_residual (the existing entry point) and the
CPU oracle, within the residual tolerance the other tests use (1e-12
relative). After its first call on the device (which looks up the array's
device address) further calls must leave the device's free memory and
PyTorch's allocated bytes unchanged, and the calling thread's current device
must be the same after a call as before it. This file is collected last so
that a run stopping at the first failure has run every other test.
"""

import numpy as np
import pytest

import oracle
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


def to_device(torch, u):
    return torch.from_numpy(np.ascontiguousarray(u).reshape(-1)).to("cuda")


def noalloc_call(torch, dev, u, out):
    nz, ny, nx = u.shape
    dt = _lib.JAC_F32 if u.dtype == np.float32 else _lib.JAC_F64
    s = torch.cuda.current_stream()
    _lib.jac_residual_dense_noalloc(dev.data_ptr(), dt, nx, ny, nz, BC, out.data_ptr(), s.cuda_stream)
    s.synchronize()
    return out.item()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_noalloc_residual_matches_context_residual_and_oracle_twice(torch_cuda, dtype):
    torch = torch_cuda
    # first call: a larger grid; second call: a smaller one, so the second
    # reads only slots it wrote itself although the array keeps the first
    # call's contents
    u1 = synth.grid_uniform01(31, 70, 45, 33).astype(dtype)
    u2 = synth.grid_uniform01(32, 20, 9, 14).astype(dtype)
    cases = [(u1, (32, 16, 11)), (u2, (8, 9, 7))]
    want = [(context_residual(u, block), oracle.residual(u, BC)) for u, block in cases]
    devs = [to_device(torch, u) for u, _ in cases]
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for (u, _), dev, (ctx, orc) in zip(cases, devs, want):
        got = noalloc_call(torch, dev, u, out)
        assert abs(got - ctx) <= 1e-12 * ctx
        assert abs(got - orc) <= 1e-12 * orc


def test_noalloc_residual_allocates_nothing_and_keeps_the_current_device(torch_cuda):
    torch = torch_cuda
    u = synth.grid_uniform01(33, 48, 40, 24)
    dev = to_device(torch, u)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    first = noalloc_call(torch, dev, u, out)  # the device's first call does the set-up
    before_free, _ = torch.cuda.mem_get_info()
    before_torch = torch.cuda.memory_allocated()
    dev_before = torch.cuda.current_device()
    vals = [noalloc_call(torch, dev, u, out) for _ in range(2)]
    assert torch.cuda.mem_get_info()[0] == before_free
    assert torch.cuda.memory_allocated() == before_torch
    assert torch.cuda.current_device() == dev_before
    assert vals[0] == first and vals[1] == first
    want = oracle.residual(u, BC)
    assert abs(first - want) <= 1e-12 * want


def test_noalloc_rejects_grids_beyond_the_scratch(torch_cuda):
    dev = torch_cuda.zeros(1, dtype=torch_cuda.float64, device="cuda")
    out = torch_cuda.zeros(1, dtype=torch_cuda.float64, device="cuda")
    # ceil(nx/32) * ceil(ny/8) = 4096 * 32 > 65536 partial slots
    with pytest.raises(_lib.JacError) as e:
        _lib.jac_residual_dense_noalloc(dev.data_ptr(), _lib.JAC_F64, 32 * 4096, 8 * 32, 1, BC, out.data_ptr())
    assert e.value.code == _lib.JAC_EINVAL
