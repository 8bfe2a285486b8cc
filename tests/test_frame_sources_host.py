"""The frame-source lists of the exact mean's work units (the units whose
exponent bounds set each tile's fixed-point frame), built by the runtime's
own code compiled for the host, against a brute-force walk over every cell
each tile's stencil reads: a unit left out of a list could put a value above
its tile's frame. Layouts: uniform and uneven block splits, tiles wider than
their blocks, ragged tile rows, units split in z."""

import ctypes
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_11819_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    d = tempfile.mkdtemp()
    out = os.path.join(d, "libframes_host.so")
    nvcc = "nvcc" if subprocess.run(["which", "nvcc"], capture_output=True).returncode == 0 else "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "host_arith", "frames_host.cu"), "-o", out], check=True, capture_output=True)
    h = ctypes.CDLL(out)
    h.host_frame_sources_check.argtypes = [ctypes.c_int] * 11 + [ctypes.c_void_p]
    h.host_frame_sources_check.restype = ctypes.c_int
    return h


def check(lib, dims, block, tw, th, zdepth, split_every, drop_last=0):
    stats = (ctypes.c_longlong * 5)()
    assert lib.host_frame_sources_check(*dims, *block, tw, th, zdepth, split_every, drop_last, stats) == 0
    return dict(zip(("units", "reads", "missing", "nolist", "longest"), stats))


LAYOUTS = [
    ((128, 128, 128), (64, 64, 64), 64, 8, 0, 0),    # the bench's shape, binary64 tiles
    ((128, 128, 128), (64, 64, 64), 64, 16, 0, 0),   # binary32 tiles
    ((100, 70, 50), (33, 40, 17), 16, 32, 0, 3),     # uneven split, units split in z
    ((96, 80, 60), (48, 40, 30), 32, 16, 12, 5),     # z depth below the block's, splits
    ((40, 24, 20), (16, 8, 10), 64, 8, 0, 2),        # tiles wider than their blocks
    ((70, 33, 21), (34, 17, 11), 32, 16, 7, 4),      # ragged rows and planes
]


@pytest.mark.parametrize("dims,block,tw,th,zdepth,split_every", LAYOUTS)
def test_every_read_cell_belongs_to_a_listed_unit(lib, dims, block, tw, th, zdepth, split_every):
    s = check(lib, dims, block, tw, th, zdepth, split_every)
    assert s["reads"] > 0 and s["nolist"] == 0
    assert s["missing"] == 0, s
    assert s["longest"] <= 256


@pytest.mark.parametrize("dims,block,tw,th,zdepth,split_every", LAYOUTS[2:4])
def test_the_check_sees_a_shortened_list(lib, dims, block, tw, th, zdepth, split_every):
    s = check(lib, dims, block, tw, th, zdepth, split_every, drop_last=1)
    assert s["missing"] > 0, s
