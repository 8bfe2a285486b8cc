"""The C-ABI library builds, loads and exports every entry point that
include/jacobi3d.h declares; argument checks that need no GPU behave.
No compute call is made here (no GPU on the CPU runner)."""

import ctypes
import os
import re

import pytest

from paper_2202_11819_gb300 import _lib, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "jacobi3d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jac_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("jac_create", "jac_iterate", "jac_residual", "jac_read", "jac_write", "jac_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = set(declared_functions())
    assert names <= set(_lib._SIGS), sorted(names - set(_lib._SIGS))


def test_strerror_and_invalid_arguments_without_gpu():
    assert _lib.jac_strerror(_lib.JAC_EINVAL) == "invalid argument"
    assert _lib.jac_strerror(_lib.JAC_ETIMEOUT) == "device wait timed out"
    with pytest.raises(_lib.JacError) as e:
        _lib.jac_create(0, 4, 4, 1, 1, 1)
    assert e.value.code == _lib.JAC_EINVAL
    with pytest.raises(_lib.JacError) as e:
        _lib.jac_create(8, 8, 8, 9, 1, 1)
    assert e.value.code == _lib.JAC_EINVAL
    with pytest.raises(_lib.JacError) as e:
        _lib.jac_create(8, 8, 8, 4, 4, 4, dtype=7)
    assert e.value.code == _lib.JAC_EINVAL
    with pytest.raises(_lib.JacError) as e:
        _lib.jac_create(8, 8, 8, 4, 4, 4, bc=(float("nan"), 0, 0, 0, 0, 0))
    assert e.value.code == _lib.JAC_EINVAL
    lib = _lib.load()
    assert lib.jac_iterate(None, 1) == _lib.JAC_EINVAL
    assert lib.jac_iterate_residual(None, 1, 1, None) == _lib.JAC_EINVAL
    assert lib.jac_destroy(None) == _lib.JAC_OK
    assert lib.jac_host_free(None) == _lib.JAC_OK
    assert lib.jac_host_free(ctypes.c_void_p(4096)) == _lib.JAC_EINVAL
    assert not lib.jac_host_alloc(0)
    assert lib.jac_host_alloc_kind(ctypes.c_void_p(4096)) == -1


def test_allocator_hook_requires_both_functions():
    lib = _lib.load()
    a = _lib.JAC_ALLOC_FN(lambda n, s, u: 0)
    assert lib.jac_set_allocator(a, _lib.JAC_FREE_FN(), None) == _lib.JAC_EINVAL
    assert lib.jac_set_allocator(_lib.JAC_ALLOC_FN(), _lib.JAC_FREE_FN(), None) == _lib.JAC_OK


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)
