"""Exact-rational Jacobi3D for tiny grids (pure Python, ``fractions``).

TEST INFRASTRUCTURE ONLY (part of the oracle). It is an independent
restatement used to pin ``jacobi_oracle.c``: the same averaging update
(the paper's Jacobi3D iteration, Section II-A, Figs. 1 and 3, two copies of
the grid per Section III-C), carried out in exact rational arithmetic, so the
only approximation anywhere is the explicit rounding step a caller asks for.

Grids are nested lists indexed [k][j][i] (x fastest), interior only; ``bc``
are the Dirichlet values of the ghost planes (-x, +x, -y, +y, -z, +z).

It also emulates the left-to-right rule operation by operation. IEEE 754
defines the result of each addition and division as the exact result rounded
once to the destination format (roundTiesToEven here). ``round_to_format``
writes that rounding out from the definition for any binary format, and
``step_sequential`` applies it after every one of the six additions and the
division by 7, in binary64 or binary32. No floating-point arithmetic of the
host takes part: every intermediate is an exact rational.
"""

from __future__ import annotations

import math
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


# ---------------------------------------------------------------------------
# IEEE 754 rounding, written from the definition
# ---------------------------------------------------------------------------

class Format:
    """A binary floating-point format: p significand bits (the leading one
    included), emin the exponent of the smallest normal number, emax of the
    largest finite one."""

    def __init__(self, p: int, emin: int, emax: int):
        self.p, self.emin, self.emax = p, emin, emax


BINARY64 = Format(53, -1022, 1023)
BINARY32 = Format(24, -126, 127)


def round_to_format(x: Fraction, fmt: Format) -> Fraction:
    """The number of ``fmt`` nearest to the rational ``x``, ties to the one
    whose last significand bit is 0 (roundTiesToEven). Results beyond the
    largest finite value raise OverflowError (the callers' inputs keep every
    sum in range). A zero result is returned as Fraction(0); the sign of zero
    is the caller's business."""
    if x == 0:
        return Fraction(0)
    a = abs(x)
    # e = floor(log2 a): 2^e <= a < 2^(e+1)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    # the quantum: the weight of the last significand bit, fixed at the
    # subnormal spacing below the normal range
    q = max(e, fmt.emin) - (fmt.p - 1)
    m = a / Fraction(2) ** q
    n = m.numerator // m.denominator
    r = m - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = n * Fraction(2) ** q
    if v >= Fraction(2) ** (fmt.emax + 1):
        raise OverflowError("result beyond the largest finite value")
    return v if x > 0 else -v


def _as_float(v: Fraction, negative_zero: bool) -> float:
    # every rounded value is exactly a binary64 number, so float() is exact
    if v == 0:
        return -0.0 if negative_zero else 0.0
    return float(v)


def add_rn(a: float, b: float, fmt: Format) -> float:
    """IEEE addition a + b in ``fmt`` (a and b are numbers of ``fmt``). An
    exact zero sum is +0 unless both operands are -0."""
    s = Fraction(a) + Fraction(b)
    if s == 0:
        return -0.0 if (math.copysign(1.0, a) < 0 and math.copysign(1.0, b) < 0) else 0.0
    return _as_float(round_to_format(s, fmt), s < 0)


def div_rn(a: float, d: float, fmt: Format) -> float:
    """IEEE division a / d in ``fmt`` (d nonzero); a zero quotient takes the
    sign of the exact quotient (or of a, for a = +-0)."""
    q = Fraction(a) / Fraction(d)
    neg = (math.copysign(1.0, a) < 0) != (d < 0)
    return _as_float(round_to_format(q, fmt), neg)


def step_sequential(u, bc, fmt: Format):
    """One iteration of the left-to-right rule in ``fmt``: the sum
    c + xm + xp + ym + yp + zm + zp taken in that order, each addition
    rounded to ``fmt``, then the sum divided by 7 and rounded. ``u`` holds
    floats that are numbers of ``fmt``; ``bc`` likewise."""
    nz, ny, nx = len(u), len(u[0]), len(u[0][0])
    out = [[[0.0] * nx for _ in range(ny)] for _ in range(nz)]
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                s = u[k][j][i]
                for (ii, jj, kk) in ((i - 1, j, k), (i + 1, j, k), (i, j - 1, k),
                                     (i, j + 1, k), (i, j, k - 1), (i, j, k + 1)):
                    s = add_rn(s, _get(u, bc, ii, jj, kk, nx, ny, nz), fmt)
                out[k][j][i] = div_rn(s, 7.0, fmt)
    return out


def iterate_sequential(u0, bc, n_iters: int, fmt: Format):
    """``n_iters`` iterations of ``step_sequential`` from the interior ``u0``
    (nz, ny, nx; its values and ``bc`` must already be numbers of ``fmt``).
    Returns nested floats."""
    bcf = [float(b) for b in bc]
    for b in bcf:
        if round_to_format(Fraction(b), fmt) != Fraction(b):
            raise ValueError("boundary value is not a number of the format")
    u = [[[float(x) for x in row] for row in plane] for plane in u0]
    for _ in range(n_iters):
        u = step_sequential(u, bcf, fmt)
    return u
