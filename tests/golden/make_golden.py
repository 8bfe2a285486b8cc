"""Writes the stored expected values under tests/golden/.

Calls only ``oracle.exact_rational`` (exact rational arithmetic) and the
``synth`` input generator; no value here comes from the CUDA path or from the
C oracle.

Every fixture is a 3 x 4 x 5 (nx, ny, nz) grid drawn from SplitMix64 seed 7
with boundary values (1, 0.25, 0, 0.5, 0, 0.125), iterated 6 times. Each line
holds the iteration number, the cell index (x fastest) and the value as a hex
float.

exact_mean_3x4x5.txt: each iteration takes the exact rational mean of a cell
  and its six face neighbours and rounds it once to the nearest binary64.
seq_rule_3x4x5.txt: each iteration forms c + xm + xp + ym + yp + zm + zp left
  to right, rounding the exact result of every addition to binary64, then
  divides by 7 and rounds (IEEE 754 operation by operation).
seq_rule_f32_3x4x5.txt: the same in binary32, from the interior rounded to
  binary32.

Run: python tests/golden/make_golden.py
"""
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import exact_rational as er  # noqa: E402
import synth  # noqa: E402

NX, NY, NZ = 3, 4, 5
SEED = 7
BC = (1.0, 0.25, 0.0, 0.5, 0.0, 0.125)
ITERS = 6


def header():
    return f"# nx={NX} ny={NY} nz={NZ} seed={SEED} bc={','.join(repr(b) for b in BC)} iters={ITERS}"


def cell_lines(it, u):
    return [f"{it} {i + NX * (j + NY * k)} {float(u[k][j][i]).hex()}"
            for k in range(NZ) for j in range(NY) for i in range(NX)]


def write(name, lines):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    u0 = synth.grid_uniform01(SEED, NX, NY, NZ)

    u = er.iterate(u0, BC, 0, round_each_step=True)
    bcf = [Fraction(b) for b in BC]
    lines = [header()]
    for it in range(1, ITERS + 1):
        u = er.step(u, bcf, round_each_step=True)
        lines += cell_lines(it, u)
    write("exact_mean_3x4x5.txt", lines)

    for name, fmt, start in (("seq_rule_3x4x5.txt", er.BINARY64, u0),
                             ("seq_rule_f32_3x4x5.txt", er.BINARY32, u0.astype(np.float32))):
        u = [[[float(x) for x in row] for row in plane] for plane in start]
        lines = [header()]
        for it in range(1, ITERS + 1):
            u = er.step_sequential(u, list(BC), fmt)
            lines += cell_lines(it, u)
        write(name, lines)


if __name__ == "__main__":
    main()
