"""jac_host_alloc: page-locked, zero-filled host buffers (huge-page backed from
64 MiB up where the kernel offers transparent huge pages), usable by the host
forms of jac_write / jac_read and by plain copies; jac_host_free releases
them."""

import ctypes

import numpy as np
import pytest

import oracle
import synth
from paper_2202_11819_gb300 import Jacobi3D, _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.load()
    yield


@pytest.mark.parametrize("nbytes", [1 << 20, (64 << 20) + 8, 1 << 30])
def test_host_alloc_is_pinned_zeroed_and_copies(nbytes):
    import torch

    torch.zeros(1, device="cuda")  # torch's CUDA state exists before it is asked about the buffer
    n = nbytes // 8
    a = _lib.host_array(n, np.float64)
    assert a.ctypes.data % 4096 == 0
    assert not a.any()
    t = torch.from_numpy(a)
    assert t.is_pinned()
    kind = _lib.jac_host_alloc_kind(a.ctypes.data)
    assert kind in (0, 1) and (kind == 0 or nbytes >= 64 << 20)
    a[:] = np.arange(n, dtype=np.float64)
    d = t.to("cuda", non_blocking=True)
    back = torch.from_numpy(_lib.host_array(n, np.float64))
    back.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    assert np.array_equal(back.numpy(), a)


def test_host_alloc_buffers_through_write_and_read():
    dims, block = (40, 24, 20), (16, 8, 10)
    u0 = synth.grid_uniform01(4, *dims)
    hin = _lib.host_array(u0.size)
    hin[:] = u0.reshape(-1)
    hout = _lib.host_array(u0.size)
    with Jacobi3D(dims, block, bc=synth.DIRICHLET_X0, mode="fused") as J:
        _lib.jac_write(J.h, hin)
        J.iterate(5)
        _lib.jac_read(J.h, hout)
    assert np.array_equal(hout.reshape(u0.shape), oracle.jacobi(u0, synth.DIRICHLET_X0, 5, oracle.RULE_EXACT))


def test_host_free_rejects_foreign_pointers():
    lib = _lib.load()
    p = _lib.jac_host_alloc(4096)
    assert lib.jac_host_free(ctypes.c_void_p(p + 64)) == _lib.JAC_EINVAL
    assert lib.jac_host_free(ctypes.c_void_p(p)) == _lib.JAC_OK
    assert lib.jac_host_free(ctypes.c_void_p(p)) == _lib.JAC_EINVAL  # already freed
