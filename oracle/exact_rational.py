"""Exact-rational Jacobi3D for tiny grids (pure Python, ``fractions``).

TEST INFRASTRUCTURE ONLY (part of the oracle). It is an independent
restatement used to pin ``jacobi_oracle.c``: the same averaging update
(the paper's Jacobi3D iteration, Section II-A, Figs. 1 and 3, two copies of
the grid per Section III-C), carried out in exact rational arithmetic, so the
only approximation anywhere is the explicit rounding step a caller asks for.

Grids are nested lists indexed [k][j][i] (x fastest), interior only; ``bc``
are the Dirichlet values of the ghost planes (-x, +x, -y, +y, -z, +z).
"""

from __future__ import annotations

from fractions import Fraction


def _get(u, bc, i, j, k, nx, ny, nz):
    if i < 0:
        return bc[0]
    if i >= nx:
        return bc[1]
    if j < 0:
        return bc[2]
    if j >= ny:
        return bc[3]
    if k < 0:
        return bc[4]
    if k >= nz:
        return bc[5]
    return u[k][j][i]


def step(u, bc, round_each_step: bool):
    """One iteration: every interior cell becomes the mean of itself and its
    six face neighbours. With ``round_each_step`` the exact mean is rounded to
    the nearest binary64 (``float(Fraction)`` is correctly rounded, ties to
    even) and stored back as an exact rational."""
    nz, ny, nx = len(u), len(u[0]), len(u[0][0])
    out = [[[None] * nx for _ in range(ny)] for _ in range(nz)]
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                s = (_get(u, bc, i, j, k, nx, ny, nz)
                     + _get(u, bc, i - 1, j, k, nx, ny, nz) + _get(u, bc, i + 1, j, k, nx, ny, nz)
                     + _get(u, bc, i, j - 1, k, nx, ny, nz) + _get(u, bc, i, j + 1, k, nx, ny, nz)
                     + _get(u, bc, i, j, k - 1, nx, ny, nz) + _get(u, bc, i, j, k + 1, nx, ny, nz))
                m = s / 7
                out[k][j][i] = Fraction(float(m)) if round_each_step else m
    return out


def iterate(u0, bc, n_iters: int, round_each_step: bool):
    """``n_iters`` iterations from the numpy/list interior ``u0`` (nz, ny, nx)."""
    bcf = [Fraction(float(b)) for b in bc]
    u = [[[Fraction(float(x)) for x in row] for row in plane] for plane in u0]
    for _ in range(n_iters):
        u = step(u, bcf, round_each_step)
    return u


def residual_sq(u, bc) -> Fraction:
    """sum over the interior of (xm + xp + ym + yp + zm + zp - 6c)^2, exactly."""
    bcf = [Fraction(float(b)) for b in bc]
    uu = [[[Fraction(x) if isinstance(x, Fraction) else Fraction(float(x)) for x in row] for row in plane] for plane in u]
    nz, ny, nx = len(uu), len(uu[0]), len(uu[0][0])
    tot = Fraction(0)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                L = (_get(uu, bcf, i - 1, j, k, nx, ny, nz) + _get(uu, bcf, i + 1, j, k, nx, ny, nz)
                     + _get(uu, bcf, i, j - 1, k, nx, ny, nz) + _get(uu, bcf, i, j + 1, k, nx, ny, nz)
                     + _get(uu, bcf, i, j, k - 1, nx, ny, nz) + _get(uu, bcf, i, j, k + 1, nx, ny, nz)
                     - 6 * uu[k][j][i])
                tot += L * L
    return tot


def to_float_grid(u):
    """Nested Fractions to nested floats (correctly rounded)."""
    return [[[float(x) for x in row] for row in plane] for plane in u]
