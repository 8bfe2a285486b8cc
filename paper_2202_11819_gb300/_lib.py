"""ctypes binding of libjacobi3d.so: the C ABI of include/jacobi3d.h with the
same names. Argument marshalling only: every step of the Jacobi iteration
runs in the library's CUDA kernels; there is no Python or CPU fallback, and a
missing or unloadable library raises.
"""

from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

from . import build as _build

JAC_OK = 0
JAC_EINVAL = -1
JAC_ENOMEM = -2
JAC_ECUDA = -3
JAC_ETIMEOUT = -4
JAC_EBUDGET = -5
JAC_ESTATE = -6

JAC_F64 = 0
JAC_F32 = 1

JAC_MODE_UNFUSED = 0
JAC_MODE_FUSED = 1
JAC_MODE_GRAPH = 2
JAC_MODE_PERSISTENT = 3
JAC_MODE_GRAPH_FUSED = 4
JAC_MODE_SPLIT = 5

JAC_ARITH_SEQ = 0
JAC_ARITH_EXACT = 1

MODES = {
    "unfused": JAC_MODE_UNFUSED,
    "fused": JAC_MODE_FUSED,
    "graph": JAC_MODE_GRAPH,
    "persistent": JAC_MODE_PERSISTENT,
    "graph_fused": JAC_MODE_GRAPH_FUSED,
    "split": JAC_MODE_SPLIT,
}


class JacError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


class jac_info_t(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int64 * 3),
        ("block", ctypes.c_int32 * 3),
        ("nblocks", ctypes.c_int32 * 3),
        ("dtype", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("arith", ctypes.c_int32),
        ("persistent_ctas", ctypes.c_int32),
        ("iterations", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("n_instances", ctypes.c_int32),
        ("tile_w", ctypes.c_int32),
        ("zdepth", ctypes.c_int32),
        ("n_units", ctypes.c_int32),
        ("n_blocks", ctypes.c_int32),
    ]


class jac_tune_t(ctypes.Structure):
    _fields_ = [
        ("tile_w", ctypes.c_int32),
        ("zdepth", ctypes.c_int32),
        ("ms_per_iter", ctypes.c_double),
        ("n_trials", ctypes.c_int32),
        ("trial_tile_w", ctypes.c_int32 * 16),
        ("trial_zdepth", ctypes.c_int32 * 16),
        ("trial_ms_per_iter", ctypes.c_double * 16),
        ("n_classes", ctypes.c_int32),
        ("class_block_x", ctypes.c_int32 * 16),
        ("class_tile_w", ctypes.c_int32 * 16),
        ("ms_per_iter_classes", ctypes.c_double),
    ]


class jac_server_stats_t(ctypes.Structure):
    _fields_ = [
        ("running", ctypes.c_int32),
        ("queued", ctypes.c_int32),
        ("finished_now", ctypes.c_int32),
        ("cell_updates", ctypes.c_int64),
        ("used_bytes", ctypes.c_int64),
        ("budget_bytes", ctypes.c_int64),
    ]


class jac_request_t(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int64),
        ("iterations", ctypes.c_int64),
        ("residual", ctypes.c_double),
        ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
        ("status", ctypes.c_int32),
    ]


JAC_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
JAC_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()

_SIGS = {
    "jac_set_allocator": ([JAC_ALLOC_FN, JAC_FREE_FN, ctypes.c_void_p], ctypes.c_int),
    "jac_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                    ctypes.c_void_p], ctypes.c_int),
    "jac_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "jac_set_mode": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "jac_set_arith": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "jac_write": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "jac_write_f32": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "jac_write_device": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32], ctypes.c_int),
    "jac_read": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "jac_read_f32": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "jac_read_device": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32], ctypes.c_int),
    "jac_iterate": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int),
    "jac_residual": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "jac_residual_device": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "jac_iterate_residual": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "jac_host_alloc": ([ctypes.c_size_t], ctypes.c_void_p),
    "jac_host_free": ([ctypes.c_void_p], ctypes.c_int),
    "jac_host_alloc_kind": ([ctypes.c_void_p], ctypes.c_int),
    "jac_sync": ([ctypes.c_void_p], ctypes.c_int),
    "jac_info": ([ctypes.c_void_p, ctypes.POINTER(jac_info_t)], ctypes.c_int),
    "jac_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "jac_last_error": ([], ctypes.c_char_p),
    "jac_set_wait_limit_ns": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int),
    "jac_debug_withhold_progress": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64], ctypes.c_int),
    "jac_create_batch": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p],
                         ctypes.c_int),
    "jac_write_instance": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "jac_write_instance_device": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.c_int32], ctypes.c_int),
    "jac_read_instance": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "jac_read_instance_device": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.c_int32], ctypes.c_int),
    "jac_residual_instances": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "jac_residual_instances_device": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "jac_set_tile": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "jac_set_tile_class": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "jac_autotune": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(jac_tune_t)], ctypes.c_int),
    "jac_storage_bytes": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                           ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "jac_create_pool": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p], ctypes.c_int),
    "jac_pool_add": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)],
                     ctypes.c_int),
    "jac_pool_remove": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "jac_pool_usage": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "jac_server_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "jac_server_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "jac_server_submit": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "jac_server_step": ([ctypes.c_void_p, ctypes.POINTER(jac_server_stats_t)], ctypes.c_int),
    "jac_server_poll": ([ctypes.c_void_p, ctypes.POINTER(jac_request_t)], ctypes.c_int),
    "jac_server_result": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "jac_server_now": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "jac_residual_dense_noalloc": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                                   ctypes.c_int),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libjacobi3d.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libjacobi3d.so not found at {path}; run paper_2202_11819_gb300.build")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, where: str) -> int:
    if rc != JAC_OK:
        lib = load()
        raise JacError(rc, where, lib.jac_last_error().decode() or lib.jac_strerror(rc).decode())
    return rc


def _host(a: np.ndarray, dtype) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


# ------------------------------------------------------------- same names as the C ABI

def jac_strerror(code: int) -> str:
    return load().jac_strerror(int(code)).decode()


def jac_last_error() -> str:
    return load().jac_last_error().decode()


def jac_set_allocator(alloc, free_fn, user=None) -> None:
    """``alloc``/``free_fn`` are JAC_ALLOC_FN / JAC_FREE_FN instances (kept
    alive by the caller) or None to restore the default."""
    lib = load()
    a = alloc if alloc is not None else JAC_ALLOC_FN()
    f = free_fn if free_fn is not None else JAC_FREE_FN()
    _check(lib.jac_set_allocator(a, f, user), "jac_set_allocator")


def jac_create(nx, ny, nz, bx, by, bz, dtype=JAC_F64, bc=(0.0,) * 6, stream=None) -> ctypes.c_void_p:
    """Returns the context handle; ``stream`` is a cudaStream_t as an int (or None)."""
    lib = load()
    h = ctypes.c_void_p()
    b = (ctypes.c_double * 6)(*[float(x) for x in bc])
    _check(lib.jac_create(ctypes.byref(h), int(nx), int(ny), int(nz), int(bx), int(by), int(bz), int(dtype),
                          b, ctypes.c_void_p(stream or 0)), "jac_create")
    return h


def jac_destroy(h) -> None:
    _check(load().jac_destroy(h), "jac_destroy")


def jac_set_mode(h, mode) -> None:
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    _check(load().jac_set_mode(h, m), "jac_set_mode")


def jac_set_arith(h, arith) -> None:
    a = {"seq": JAC_ARITH_SEQ, "exact": JAC_ARITH_EXACT}[arith] if isinstance(arith, str) else int(arith)
    _check(load().jac_set_arith(h, a), "jac_set_arith")


def jac_write(h, host: np.ndarray) -> None:
    a = _host(host, np.float64)
    _check(load().jac_write(h, a.ctypes.data, a.size), "jac_write")


def jac_write_f32(h, host: np.ndarray) -> None:
    a = _host(host, np.float32)
    _check(load().jac_write_f32(h, a.ctypes.data, a.size), "jac_write_f32")


def jac_write_device(h, dev_ptr: int, n_cells: int, dtype: int) -> None:
    _check(load().jac_write_device(h, ctypes.c_void_p(dev_ptr), int(n_cells), int(dtype)), "jac_write_device")


def jac_read(h, out: np.ndarray) -> np.ndarray:
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array")
    _check(load().jac_read(h, out.ctypes.data, out.size), "jac_read")
    return out


def jac_read_f32(h, out: np.ndarray) -> np.ndarray:
    if out.dtype != np.float32 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float32 array")
    _check(load().jac_read_f32(h, out.ctypes.data, out.size), "jac_read_f32")
    return out


def jac_read_device(h, dev_ptr: int, n_cells: int, dtype: int) -> None:
    _check(load().jac_read_device(h, ctypes.c_void_p(dev_ptr), int(n_cells), int(dtype)), "jac_read_device")


def jac_iterate(h, n_iters: int) -> None:
    _check(load().jac_iterate(h, int(n_iters)), "jac_iterate")


def jac_residual(h) -> float:
    r = ctypes.c_double()
    _check(load().jac_residual(h, ctypes.byref(r)), "jac_residual")
    return r.value


def jac_residual_device(h, dev_ptr: int) -> None:
    _check(load().jac_residual_device(h, ctypes.c_void_p(dev_ptr)), "jac_residual_device")


def jac_host_alloc(nbytes: int) -> int:
    p = load().jac_host_alloc(int(nbytes))
    if not p:
        raise JacError(JAC_ENOMEM, "jac_host_alloc", jac_last_error())
    return p


def jac_host_free(ptr: int) -> None:
    _check(load().jac_host_free(ctypes.c_void_p(ptr)), "jac_host_free")


def jac_host_alloc_kind(ptr: int) -> int:
    return load().jac_host_alloc_kind(ctypes.c_void_p(ptr))


def host_array(n: int, dtype=np.float64) -> np.ndarray:
    """A numpy array of n values in jac_host_alloc memory (freed with the
    last array or tensor viewing it)."""
    dt = np.dtype(dtype)
    nbytes = max(1, n * dt.itemsize)
    ptr = jac_host_alloc(nbytes)
    buf = (ctypes.c_char * nbytes).from_address(ptr)
    weakref.finalize(buf, jac_host_free, ptr)
    return np.frombuffer(buf, dtype=dt, count=n)


def jac_iterate_residual(h, n_iters: int, every: int, dev_ptr: int) -> None:
    _check(load().jac_iterate_residual(h, int(n_iters), int(every), ctypes.c_void_p(dev_ptr)),
           "jac_iterate_residual")


def jac_sync(h) -> None:
    _check(load().jac_sync(h), "jac_sync")


def jac_info(h) -> dict:
    info = jac_info_t()
    _check(load().jac_info(h, ctypes.byref(info)), "jac_info")
    return {
        "dims": tuple(info.dims),
        "block": tuple(info.block),
        "nblocks": tuple(info.nblocks),
        "dtype": info.dtype,
        "mode": info.mode,
        "arith": info.arith,
        "persistent_ctas": info.persistent_ctas,
        "iterations": info.iterations,
        "device_bytes": info.device_bytes,
        "kernel_launches": info.kernel_launches,
        "n_instances": info.n_instances,
        "tile_w": info.tile_w,
        "zdepth": info.zdepth,
        "n_units": info.n_units,
        "n_blocks": info.n_blocks,
    }


def jac_create_batch(dims, bx, by, bz, dtype=JAC_F64, bcs=None, stream=None) -> ctypes.c_void_p:
    """``dims``: list of (nx, ny, nz); ``bcs``: list of 6-tuples (one per grid)."""
    lib = load()
    n = len(dims)
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64).reshape(n, 3))
    b = np.ascontiguousarray(np.asarray(bcs if bcs is not None else [(0.0,) * 6] * n, dtype=np.float64).reshape(n, 6))
    h = ctypes.c_void_p()
    _check(lib.jac_create_batch(ctypes.byref(h), n, d.ctypes.data, int(bx), int(by), int(bz), int(dtype),
                                b.ctypes.data, ctypes.c_void_p(stream or 0)), "jac_create_batch")
    return h


def jac_write_instance(h, i: int, host: np.ndarray) -> None:
    a = _host(host, np.float64)
    _check(load().jac_write_instance(h, int(i), a.ctypes.data, a.size), "jac_write_instance")


def jac_write_instance_device(h, i: int, dev_ptr: int, n_cells: int, dtype: int) -> None:
    _check(load().jac_write_instance_device(h, int(i), ctypes.c_void_p(dev_ptr), int(n_cells), int(dtype)),
           "jac_write_instance_device")


def jac_read_instance(h, i: int, out: np.ndarray) -> np.ndarray:
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array")
    _check(load().jac_read_instance(h, int(i), out.ctypes.data, out.size), "jac_read_instance")
    return out


def jac_read_instance_device(h, i: int, dev_ptr: int, n_cells: int, dtype: int) -> None:
    _check(load().jac_read_instance_device(h, int(i), ctypes.c_void_p(dev_ptr), int(n_cells), int(dtype)),
           "jac_read_instance_device")


def jac_residual_instances(h, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _check(load().jac_residual_instances(h, out.ctypes.data), "jac_residual_instances")
    return out


def jac_residual_instances_device(h, dev_ptr: int) -> None:
    _check(load().jac_residual_instances_device(h, ctypes.c_void_p(dev_ptr)), "jac_residual_instances_device")


def jac_set_tile(h, tile_w: int, zdepth: int) -> None:
    _check(load().jac_set_tile(h, int(tile_w), int(zdepth)), "jac_set_tile")


def jac_set_tile_class(h, block_x: int, tile_w: int) -> None:
    _check(load().jac_set_tile_class(h, int(block_x), int(tile_w)), "jac_set_tile_class")


def jac_autotune(h, trial_iters: int) -> dict:
    r = jac_tune_t()
    _check(load().jac_autotune(h, int(trial_iters), ctypes.byref(r)), "jac_autotune")
    n = min(r.n_trials, 16)
    out = {"tile_w": r.tile_w, "zdepth": r.zdepth, "ms_per_iter": r.ms_per_iter,
           "trials": [(r.trial_tile_w[i], r.trial_zdepth[i], r.trial_ms_per_iter[i]) for i in range(n)],
           "n_trials": r.n_trials}
    if r.n_classes:
        out["classes"] = [(r.class_block_x[i], r.class_tile_w[i]) for i in range(min(r.n_classes, 16))]
        out["ms_per_iter_classes"] = r.ms_per_iter_classes
    return out


def _i64x3(dims):
    return (ctypes.c_int64 * 3)(*[int(v) for v in dims])


def _f64x6(bc):
    return (ctypes.c_double * 6)(*[float(v) for v in bc])


def jac_storage_bytes(dims, bx, by, bz, dtype=JAC_F64) -> int:
    out = ctypes.c_int64()
    _check(load().jac_storage_bytes(_i64x3(dims), int(bx), int(by), int(bz), int(dtype), ctypes.byref(out)),
           "jac_storage_bytes")
    return out.value


def jac_create_pool(dtype, capacity_bytes, max_grids, bx, by, bz, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().jac_create_pool(ctypes.byref(h), int(dtype), int(capacity_bytes), int(max_grids), int(bx),
                                  int(by), int(bz), ctypes.c_void_p(stream or 0)), "jac_create_pool")
    return h


def jac_pool_add(h, dims, bc) -> int:
    slot = ctypes.c_int32()
    _check(load().jac_pool_add(h, _i64x3(dims), _f64x6(bc), ctypes.byref(slot)), "jac_pool_add")
    return slot.value


def jac_pool_remove(h, slot: int) -> None:
    _check(load().jac_pool_remove(h, int(slot)), "jac_pool_remove")


def jac_pool_usage(h) -> tuple:
    u, c, g = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(load().jac_pool_usage(h, ctypes.byref(u), ctypes.byref(c), ctypes.byref(g)), "jac_pool_usage")
    return u.value, c.value, g.value


def jac_server_create(budget_bytes, max_active, bx, by, bz, chunk_iters) -> ctypes.c_void_p:
    s = ctypes.c_void_p()
    _check(load().jac_server_create(ctypes.byref(s), int(budget_bytes), int(max_active), int(bx), int(by), int(bz),
                                    int(chunk_iters)), "jac_server_create")
    return s


def jac_server_destroy(s) -> None:
    _check(load().jac_server_destroy(s), "jac_server_destroy")


def jac_server_submit(s, dims, dtype, bc, init: np.ndarray, tol: float, max_iters: int) -> int:
    a = _host(init, np.float64)
    rid = ctypes.c_int64()
    _check(load().jac_server_submit(s, _i64x3(dims), int(dtype), _f64x6(bc), a.ctypes.data, float(tol),
                                    int(max_iters), ctypes.byref(rid)), "jac_server_submit")
    return rid.value


def jac_server_step(s) -> dict:
    st = jac_server_stats_t()
    _check(load().jac_server_step(s, ctypes.byref(st)), "jac_server_step")
    return {k: getattr(st, k) for k, _ in jac_server_stats_t._fields_}


def jac_server_poll(s):
    r = jac_request_t()
    rc = load().jac_server_poll(s, ctypes.byref(r))
    if rc == JAC_ESTATE:
        return None
    _check(rc, "jac_server_poll")
    return {k: getattr(r, k) for k, _ in jac_request_t._fields_}


def jac_server_result(s, req_id: int, out: np.ndarray | None) -> np.ndarray | None:
    if out is None:
        _check(load().jac_server_result(s, int(req_id), None, 0), "jac_server_result")
        return None
    _check(load().jac_server_result(s, int(req_id), out.ctypes.data, out.size), "jac_server_result")
    return out


def jac_server_now(s) -> float:
    t = ctypes.c_double()
    _check(load().jac_server_now(s, ctypes.byref(t)), "jac_server_now")
    return t.value


def jac_set_wait_limit_ns(h, ns: int) -> None:
    _check(load().jac_set_wait_limit_ns(h, int(ns)), "jac_set_wait_limit_ns")


def jac_debug_withhold_progress(h, block: int, after_iter: int) -> None:
    _check(load().jac_debug_withhold_progress(h, int(block), int(after_iter)), "jac_debug_withhold_progress")


def jac_residual_dense_noalloc(dev_u: int, dtype: int, nx: int, ny: int, nz: int, bc, dev_out: int,
                               stream=None) -> None:
    """Residual of a caller-held dense device grid into the device double at
    ``dev_out``; allocates nothing (scratch is a fixed static device array)."""
    b = (ctypes.c_double * 6)(*[float(x) for x in bc])
    rc = load().jac_residual_dense_noalloc(ctypes.c_void_p(dev_u), int(dtype), int(nx), int(ny), int(nz), b,
                                           ctypes.c_void_p(dev_out), ctypes.c_void_p(stream or 0))
    if rc != JAC_OK:
        raise JacError(rc, "jac_residual_dense_noalloc", jac_strerror(rc))
