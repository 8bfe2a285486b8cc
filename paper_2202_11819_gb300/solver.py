"""Convenience wrapper over the C ABI: one ``Jacobi3D`` object per context.

PyTorch provides the device memory (the library's allocations are routed to
PyTorch's caching allocator through ``jac_set_allocator``) and the stream
(the context runs on ``torch.cuda.current_stream()`` unless given one).
Everything else is a call into libjacobi3d.
"""

from __future__ import annotations

import numpy as np

from . import _lib

_TORCH_HOOK = None  # keeps the ctypes callbacks alive


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through PyTorch's caching
    allocator (contexts created afterwards)."""
    global _TORCH_HOOK
    if not enable:
        _lib.jac_set_allocator(None, None)
        _TORCH_HOOK = None
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0)))
        except Exception:  # noqa: BLE001 - reported to the library as NULL
            return 0

    def _free(ptr, nbytes, stream, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:  # noqa: BLE001
            pass

    a = _lib.JAC_ALLOC_FN(_alloc)
    f = _lib.JAC_FREE_FN(_free)
    _lib.jac_set_allocator(a, f)
    _TORCH_HOOK = (a, f)


class Jacobi3D:
    """A global grid of ``dims`` (nx, ny, nz) split into blocks of ``block``
    (bx, by, bz) with Dirichlet values ``bc`` (-x, +x, -y, +y, -z, +z)."""

    def __init__(self, dims, block, dtype: str = "f64", bc=(1.0, 0.0, 0.0, 0.0, 0.0, 0.0), stream=None,
                 mode: str = "persistent", arith: str | None = None):
        nx, ny, nz = (int(v) for v in dims)
        bx, by, bz = (int(v) for v in block)
        self.dims = (nx, ny, nz)
        self.dtype = dtype
        self._dt = _lib.JAC_F32 if dtype == "f32" else _lib.JAC_F64
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except Exception:  # noqa: BLE001
                stream = None
        self.h = _lib.jac_create(nx, ny, nz, bx, by, bz, self._dt, bc, stream)
        self.set_mode(mode)
        if arith is not None:
            self.set_arith(arith)

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None) is not None:
            _lib.jac_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    # -- configuration
    def set_mode(self, mode):
        _lib.jac_set_mode(self.h, mode)

    def set_arith(self, arith):
        _lib.jac_set_arith(self.h, arith)

    def info(self) -> dict:
        return _lib.jac_info(self.h)

    # -- data
    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)

    def write(self, u: np.ndarray):
        if self.dtype == "f32" and u.dtype == np.float32:
            _lib.jac_write_f32(self.h, u)
        else:
            _lib.jac_write(self.h, u)

    def write_device(self, tensor):
        """From a contiguous CUDA tensor of the context's dtype."""
        _lib.jac_write_device(self.h, tensor.data_ptr(), tensor.numel(), self._dt)

    def read(self, dtype=np.float64) -> np.ndarray:
        if dtype == np.float32:
            return _lib.jac_read_f32(self.h, np.empty(self.shape, dtype=np.float32))
        return _lib.jac_read(self.h, np.empty(self.shape, dtype=np.float64))

    def read_device(self, tensor):
        import torch

        dt = _lib.JAC_F32 if tensor.dtype == torch.float32 else _lib.JAC_F64
        _lib.jac_read_device(self.h, tensor.data_ptr(), tensor.numel(), dt)
        return tensor

    # -- compute
    def iterate(self, n: int):
        _lib.jac_iterate(self.h, n)

    def residual(self) -> float:
        return _lib.jac_residual(self.h)

    def residual_device(self, out_tensor):
        _lib.jac_residual_device(self.h, out_tensor.data_ptr())
        return out_tensor

    def iterate_residual(self, n: int, every: int, out_tensor):
        """n iterations and rho of the grid before every `every`-th of them:
        out_tensor (device float64, at least ceil(n / every) values) gets
        rho(u^(k0 + j * every)), j = 0, 1, ..."""
        need = -(-int(n) // int(every)) if n > 0 and every > 0 else 0
        if str(out_tensor.dtype) != "torch.float64" or not out_tensor.is_cuda or not out_tensor.is_contiguous():
            raise ValueError("out_tensor must be a contiguous float64 CUDA tensor")
        if out_tensor.numel() < need:
            raise ValueError(f"out_tensor holds {out_tensor.numel()} values, {need} needed")
        _lib.jac_iterate_residual(self.h, n, every, out_tensor.data_ptr())
        return out_tensor

    def sync(self):
        _lib.jac_sync(self.h)


class Jacobi3DBatch:
    """Several independent grids in one context: one pool, one block table,
    advanced together by every launch. ``dims`` is a list of (nx, ny, nz),
    ``bcs`` a list of 6-tuples."""

    def __init__(self, dims, block, dtype: str = "f64", bcs=None, stream=None, mode: str = "persistent",
                 arith: str | None = None):
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.dtype = dtype
        self._dt = _lib.JAC_F32 if dtype == "f32" else _lib.JAC_F64
        if bcs is None:
            bcs = [(1.0, 0.0, 0.0, 0.0, 0.0, 0.0)] * len(self.dims)
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except Exception:  # noqa: BLE001
                stream = None
        bx, by, bz = (int(v) for v in block)
        self.h = _lib.jac_create_batch(self.dims, bx, by, bz, self._dt, bcs, stream)
        _lib.jac_set_mode(self.h, mode)
        if arith is not None:
            _lib.jac_set_arith(self.h, arith)

    def close(self):
        if getattr(self, "h", None) is not None:
            _lib.jac_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def shape(self, i):
        nx, ny, nz = self.dims[i]
        return (nz, ny, nx)

    def write(self, i, u):
        _lib.jac_write_instance(self.h, i, u)

    def read(self, i):
        return _lib.jac_read_instance(self.h, i, np.empty(self.shape(i), dtype=np.float64))

    def iterate(self, n):
        _lib.jac_iterate(self.h, n)

    def residuals(self):
        return _lib.jac_residual_instances(self.h, len(self.dims))

    def set_mode(self, mode):
        _lib.jac_set_mode(self.h, mode)

    def set_tile(self, tile_w, zdepth):
        _lib.jac_set_tile(self.h, tile_w, zdepth)

    def set_tile_class(self, block_x, tile_w):
        _lib.jac_set_tile_class(self.h, block_x, tile_w)

    def autotune(self, trial_iters=4):
        return _lib.jac_autotune(self.h, trial_iters)

    def info(self):
        return _lib.jac_info(self.h)

    def sync(self):
        _lib.jac_sync(self.h)
