"""Jacobi3D oracle (CPU, plain, slow, obviously correct).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (``paper_2202_11819_gb300``) never imports it, and it never
imports the product path: the two share no code.

The arithmetic lives in ``jacobi_oracle.c`` (binary64, undecomposed global
grid with a one-cell Dirichlet ghost frame; see the header comment there for
the readings of the paper it follows). ``exact_rational.py`` is a second,
independent, exact-rational implementation for tiny grids used to pin it.

Arrays are numpy arrays of shape (nz, ny, nx): x is the fastest axis.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RULE_SEQ = 0    # left-to-right binary64 sum, then / 7 (correctly rounded)
RULE_EXACT = 1  # exact sum of the seven values / 7, rounded once


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP if available). Returns its path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, dp = ctypes.c_int64, ctypes.c_void_p
        lib.orc_jacobi_f64.argtypes = [i64, i64, i64, dp, dp, i64, dp, ctypes.c_int]
        lib.orc_jacobi_f64.restype = ctypes.c_int
        lib.orc_jacobi_f32.argtypes = [i64, i64, i64, dp, dp, i64, dp]
        lib.orc_jacobi_f32.restype = ctypes.c_int
        lib.orc_residual_f64.argtypes = [i64, i64, i64, dp, dp, dp]
        lib.orc_residual_f64.restype = ctypes.c_int
        lib.orc_residual_f32.argtypes = [i64, i64, i64, dp, dp, dp]
        lib.orc_residual_f32.restype = ctypes.c_int
        lib.orc_exact_mean7.argtypes = [dp]
        lib.orc_exact_mean7.restype = ctypes.c_double
        lib.orc_exact_laplacian.argtypes = [ctypes.c_double, dp]
        lib.orc_exact_laplacian.restype = ctypes.c_double
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _bc_array(bc) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(bc, dtype=np.float64).reshape(6))
    return b


def jacobi(u0: np.ndarray, bc, n_iters: int, rule: int = RULE_SEQ) -> np.ndarray:
    """``n_iters`` binary64 Jacobi iterations of the interior ``u0`` (nz, ny, nx)
    with Dirichlet ghost values ``bc`` = (-x, +x, -y, +y, -z, +z)."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    nz, ny, nx = u0.shape
    out = np.empty_like(u0)
    b = _bc_array(bc)
    rc = _load().orc_jacobi_f64(nx, ny, nz, _ptr(b), _ptr(u0), int(n_iters), _ptr(out), int(rule))
    if rc != 0:
        raise RuntimeError(f"orc_jacobi_f64 failed: {rc}")
    return out


def jacobi_f32(u0: np.ndarray, bc, n_iters: int) -> np.ndarray:
    """``n_iters`` binary32 Jacobi iterations (bc rounded to binary32)."""
    u0 = np.ascontiguousarray(u0, dtype=np.float32)
    nz, ny, nx = u0.shape
    out = np.empty_like(u0)
    b = _bc_array(bc)
    rc = _load().orc_jacobi_f32(nx, ny, nz, _ptr(b), _ptr(u0), int(n_iters), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_jacobi_f32 failed: {rc}")
    return out


def residual(u: np.ndarray, bc) -> float:
    """rho(u) = sqrt(sum L^2), L = xm+xp+ym+yp+zm+zp-6c exact then rounded."""
    b = _bc_array(bc)
    rho = np.zeros(1, dtype=np.float64)
    if u.dtype == np.float32:
        u = np.ascontiguousarray(u)
        nz, ny, nx = u.shape
        rc = _load().orc_residual_f32(nx, ny, nz, _ptr(b), _ptr(u), _ptr(rho))
    else:
        u = np.ascontiguousarray(u, dtype=np.float64)
        nz, ny, nx = u.shape
        rc = _load().orc_residual_f64(nx, ny, nz, _ptr(b), _ptr(u), _ptr(rho))
    if rc != 0:
        raise RuntimeError(f"orc_residual failed: {rc}")
    return float(rho[0])


def exact_mean7(values) -> float:
    """Correctly rounded mean of seven doubles (exposed for exactness pins)."""
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(7))
    return float(_load().orc_exact_mean7(_ptr(v)))


def exact_laplacian(c: float, nb) -> float:
    """xm+xp+ym+yp+zm+zp-6c, exact then rounded once (exposed for pins)."""
    v = np.ascontiguousarray(np.asarray(nb, dtype=np.float64).reshape(6))
    return float(_load().orc_exact_laplacian(float(c), _ptr(v)))


def num_threads() -> int:
    """Host threads the oracle's OpenMP loops use."""
    return int(_load().orc_num_threads())
