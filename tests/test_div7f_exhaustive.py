"""The binary32 division by 7 used by the CUDA path (a two-word reciprocal
and one fused multiply-add, with an exact integer path for tiny values),
compiled for the host and compared bit for bit with the correctly rounded
quotient for every finite binary32 value (about 4.3e9 cases, OpenMP)."""

import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_11819_gb300", "csrc")


@pytest.mark.slow
def test_div7f_is_correctly_rounded_for_every_finite_float():
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "div7f_exhaustive")
    nvcc = "nvcc" if subprocess.run(["which", "nvcc"], capture_output=True).returncode == 0 else "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fopenmp,-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "host_arith", "div7f_exhaustive.cu"), "-o", exe], check=True,
                   capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad=0" in r.stdout
