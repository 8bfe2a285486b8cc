"""The oracle against stored exact-rational iterates (tests/golden/).

The fixtures are written by tests/golden/make_golden.py from
oracle/exact_rational.py alone: the correctly rounded mean, and the
left-to-right rule emulated operation by operation (every addition and the
division by 7 rounded from its exact result, IEEE 754) in binary64 and
binary32.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NX, NY, NZ = 3, 4, 5
BC = (1.0, 0.25, 0.0, 0.5, 0.0, 0.125)


def load(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        header = f.readline()
        for line in f:
            it, cell, hx = line.split()
            rows.setdefault(int(it), {})[int(cell)] = float.fromhex(hx)
    assert "nx=3 ny=4 nz=5 seed=7" in header
    return rows


def _run(kind, u0, it):
    if kind == "exact":
        return oracle.jacobi(u0, BC, it, oracle.RULE_EXACT)
    if kind == "seq":
        return oracle.jacobi(u0, BC, it, oracle.RULE_SEQ)
    return oracle.jacobi_f32(u0.astype(np.float32), BC, it).astype(np.float64)


@pytest.mark.parametrize("name,kind", [("exact_mean_3x4x5.txt", "exact"),
                                       ("seq_rule_3x4x5.txt", "seq"),
                                       ("seq_rule_f32_3x4x5.txt", "f32")])
def test_oracle_matches_stored_rational_iterates(name, kind):
    rows = load(name)
    assert sorted(rows) == list(range(1, 7))
    u0 = synth.grid_uniform01(7, NX, NY, NZ)
    for it, cells in rows.items():
        got = _run(kind, u0, it).reshape(-1)
        want = np.array([cells[c] for c in range(NX * NY * NZ)])
        assert np.array_equal(got, want), f"{name}: iteration {it}"
