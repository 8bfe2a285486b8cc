"""Planted mistakes in the oracle must fail at least one pin.

Each mutant is the oracle's C source compiled with -DORC_MUTANT=n into a
temporary directory (the real library is untouched). The pins of
``test_oracle_pins`` are then run against it; the mutant must be caught.
"""

import ctypes
import os
import subprocess
import tempfile

import pytest

import oracle
import synth
from tests import test_oracle_pins as pins

MUTANTS = {
    1: "sequential sum drops the +z neighbour",
    2: "boundary values of the -x and +x faces swapped",
    3: "-y neighbour read along x (transposed index)",
    4: "correctly rounded mean truncates instead of rounding",
    5: "residual adds 6c instead of subtracting it",
    6: "sequential mean divides by 6",
    7: "sequential sum adds xm + xp first (reordered)",
    8: "sequential mean multiplies by fl(1/7) instead of dividing by 7",
    9: "binary32 mean multiplies by fl(1/7) instead of dividing by 7",
}

CHECKS = [
    lambda: pins.test_sine_mode_decays_by_closed_form_factor(oracle.RULE_SEQ, (6, 5, 7), (1, 2, 3)),
    lambda: pins.test_sine_mode_decays_by_closed_form_factor(oracle.RULE_EXACT, (6, 5, 7), (1, 2, 3)),
    lambda: pins.test_exact_rule_equals_rational_mean_rounded_each_step((3, 4, 5)),
    lambda: pins.test_seq_rule_within_roundoff_of_exact_rational((3, 4, 5)),
    lambda: pins.test_limit_is_dense_dirichlet_solution(oracle.RULE_SEQ, synth.DIRICHLET_X0),
    lambda: pins.test_limit_is_dense_dirichlet_solution(oracle.RULE_EXACT, synth.DIRICHLET_X0),
    lambda: pins.test_residual_of_sine_mode_closed_form((6, 5, 7), (1, 2, 3)),
    lambda: pins.test_exact_mean7_adversarial(),
    lambda: pins.test_seq_rule_equals_per_operation_rounding((3, 4, 5)),
    lambda: pins.test_f32_equals_per_operation_rounding((3, 4, 5)),
]


def _build_mutant(n, d):
    src = os.path.join(os.path.dirname(oracle.__file__), "jacobi_oracle.c")
    out = os.path.join(d, f"liboracle_m{n}.so")
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", f"-DORC_MUTANT={n}",
                    "-o", out, src], check=True, capture_output=True)
    return out


@pytest.mark.parametrize("n", sorted(MUTANTS))
def test_mutant_is_caught(n, monkeypatch):
    real = oracle._load()
    with tempfile.TemporaryDirectory() as d:
        lib = ctypes.CDLL(_build_mutant(n, d))
        for name in ("orc_jacobi_f64", "orc_jacobi_f32", "orc_residual_f64", "orc_residual_f32",
                     "orc_exact_mean7", "orc_exact_laplacian", "orc_num_threads"):
            getattr(lib, name).argtypes = getattr(real, name).argtypes
            getattr(lib, name).restype = getattr(real, name).restype
        monkeypatch.setattr(oracle, "_lib", lib)
        caught = 0
        for check in CHECKS:
            try:
                check()
            except AssertionError:
                caught += 1
        assert caught > 0, f"mutant {n} ({MUTANTS[n]}) passed every pin"


def test_unmutated_oracle_passes_the_same_checks():
    for check in CHECKS:
        check()
