"""Writes the stored expected values under tests/golden/.

Calls only ``oracle.exact_rational`` (exact rational arithmetic) and the
``synth`` input generator; no value here comes from the CUDA path.

exact_mean_3x4x5.txt: a 3 x 4 x 5 (nx, ny, nz) grid drawn from SplitMix64
seed 7, boundary values (1, 0.25, 0, 0.5, 0, 0.125), iterated 6 times where
each iteration takes the exact rational mean of a cell and its six face
neighbours and rounds it to the nearest binary64. Each line holds the
iteration number, the cell index (x fastest) and the value as a hex float.

Run: python tests/golden/make_golden.py
"""
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact_rational as er  # noqa: E402
import synth  # noqa: E402

NX, NY, NZ = 3, 4, 5
SEED = 7
BC = (1.0, 0.25, 0.0, 0.5, 0.0, 0.125)
ITERS = 6


def main():
    u0 = synth.grid_uniform01(SEED, NX, NY, NZ)
    u = er.iterate(u0, BC, 0, round_each_step=True)
    bcf = [Fraction(b) for b in BC]
    lines = [f"# nx={NX} ny={NY} nz={NZ} seed={SEED} bc={','.join(repr(b) for b in BC)} iters={ITERS}"]
    for it in range(1, ITERS + 1):
        u = er.step(u, bcf, round_each_step=True)
        for k in range(NZ):
            for j in range(NY):
                for i in range(NX):
                    lines.append(f"{it} {i + NX * (j + NY * k)} {float(u[k][j][i]).hex()}")
    with open(os.path.join(HERE, "exact_mean_3x4x5.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
