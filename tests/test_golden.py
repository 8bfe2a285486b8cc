"""The oracle against stored exact-rational iterates (tests/golden/)."""
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "exact_mean_3x4x5.txt")


def load():
    rows = {}
    with open(GOLDEN) as f:
        header = f.readline()
        for line in f:
            it, cell, hx = line.split()
            rows.setdefault(int(it), {})[int(cell)] = float.fromhex(hx)
    return header, rows


def test_exact_rule_matches_stored_rational_iterates():
    header, rows = load()
    assert "nx=3 ny=4 nz=5 seed=7" in header
    nx, ny, nz = 3, 4, 5
    bc = (1.0, 0.25, 0.0, 0.5, 0.0, 0.125)
    u0 = synth.grid_uniform01(7, nx, ny, nz)
    for it, cells in rows.items():
        got = oracle.jacobi(u0, bc, it, oracle.RULE_EXACT).reshape(-1)
        want = np.array([cells[c] for c in range(nx * ny * nz)])
        assert np.array_equal(got, want), f"iteration {it}"
