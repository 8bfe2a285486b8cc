"""Pins of the CPU oracle to facts fixed by mathematics, not by the oracle.

Each test is chosen so that a plausible mistake in the oracle (a dropped or
doubled neighbour, a wrong sign, a boundary value on the wrong face, a
transposed axis, a wrong rounding) fails at least one of them:

- constant fields are fixed points (exact for the correctly rounded mean);
- separable sine modes decay by the closed-form factor per iteration;
- exact-rational brute force on tiny grids (Python ``fractions``): the
  correctly rounded mean against the rational mean rounded once, and the
  left-to-right rule (binary64 and binary32) against an emulation that rounds
  the exact result of every addition and of the division, as IEEE 754
  defines each operation;
- the iteration's limit equals a dense linear solve of the discrete
  Dirichlet problem built here from the problem statement;
- maximum principle, monotone residual decay, the asymptotic rate;
- the residual of a sine mode in closed form;
- axis-permutation covariance.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact_rational as er
import synth

U = 2.0 ** -53  # unit roundoff of binary64


def rand_grid(seed, nx, ny, nz):
    return synth.grid_uniform01(seed, nx, ny, nz).copy()


# ---------------------------------------------------------------- P1 fixed point
@pytest.mark.parametrize("c", [0.0, 0.5, 1.0, 3.0, 0.75])
@pytest.mark.parametrize("rule", [oracle.RULE_SEQ, oracle.RULE_EXACT])
def test_constant_field_is_fixed_point(c, rule):
    u0 = np.full((5, 4, 6), c)
    out = oracle.jacobi(u0, [c] * 6, 7, rule)
    assert np.array_equal(out, u0)


@pytest.mark.parametrize("c", [0.1, 1.0 / 3.0, math.pi, 1e-300, 2.0 ** -1070])
def test_constant_field_fixed_point_exact_rule_any_value(c):
    # the correctly rounded mean of seven copies of c is c for every double
    u0 = np.full((3, 4, 5), c)
    out = oracle.jacobi(u0, [c] * 6, 3, oracle.RULE_EXACT)
    assert np.array_equal(out, u0)


# ---------------------------------------------------------------- P2 eigenmode
def sine_mode(n, m):
    nx, ny, nz = n
    mx, my, mz = m
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    sx = np.sin(np.pi * mx * (i + 1) / (nx + 1))
    sy = np.sin(np.pi * my * (j + 1) / (ny + 1))
    sz = np.sin(np.pi * mz * (k + 1) / (nz + 1))
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def mode_factor(n, m):
    return (1.0 + 2.0 * sum(math.cos(math.pi * mm / (nn + 1)) for nn, mm in zip(n, m))) / 7.0


@pytest.mark.parametrize("rule", [oracle.RULE_SEQ, oracle.RULE_EXACT])
@pytest.mark.parametrize("n,m", [((6, 5, 7), (1, 2, 3)), ((9, 4, 3), (2, 1, 1)), ((5, 5, 5), (3, 3, 1))])
def test_sine_mode_decays_by_closed_form_factor(rule, n, m):
    u0 = sine_mode(n, m)
    lam = mode_factor(n, m)
    k = 20
    out = oracle.jacobi(u0, [0.0] * 6, k, rule)
    expect = lam ** k * u0
    # each iteration adds at most a few units of roundoff of max|u|
    err = np.max(np.abs(out - expect))
    assert err <= k * 8 * U * np.max(np.abs(u0)) + 1e-300
    # and the decay is not trivially satisfied
    assert np.max(np.abs(out)) > 0.5 * abs(lam) ** k * np.max(np.abs(u0))


# ---------------------------------------------------------------- P3 brute force
BC_MIXED = (1.0, 0.25, 0.0, 0.5, 0.0, 0.125)


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 5)])
def test_exact_rule_equals_rational_mean_rounded_each_step(shape):
    nx, ny, nz = shape
    u0 = rand_grid(3, nx, ny, nz)
    ref = er.iterate(u0, BC_MIXED, 0, round_each_step=True)
    for k in range(1, 5):
        ref = er.step(ref, [Fraction(b) for b in BC_MIXED], round_each_step=True)
        got = oracle.jacobi(u0, BC_MIXED, k, oracle.RULE_EXACT)
        assert np.array_equal(got, np.array(er.to_float_grid(ref))), f"iteration {k}"


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 5)])
def test_seq_rule_within_roundoff_of_exact_rational(shape):
    nx, ny, nz = shape
    u0 = rand_grid(4, nx, ny, nz)
    exact = er.iterate(u0, BC_MIXED, 0, round_each_step=False)
    bcf = [Fraction(b) for b in BC_MIXED]
    M = 1.0  # every value and boundary lies in [0, 1]
    for k in range(1, 6):
        exact = er.step(exact, bcf, round_each_step=False)
        got = oracle.jacobi(u0, BC_MIXED, k, oracle.RULE_SEQ)
        worst = max(abs(Fraction(float(got[kk, jj, ii])) - exact[kk][jj][ii])
                    for kk in range(nz) for jj in range(ny) for ii in range(nx))
        # per step: six partial sums rounded (each <= 7M) then a rounded quotient
        per_step = (sum(0.5 * 2.0 ** -52 * (t + 1) for t in range(1, 7)) / 7 + 0.5 * 2.0 ** -53) * M
        assert float(worst) <= k * per_step
        if k == 1:
            assert float(worst) > 0.0  # rounding did happen: the test is not vacuous


# ------------------------------------------ P3' per-operation rounding (IEEE 754)
def _signs_equal(a, b):
    return np.array_equal(np.signbit(a), np.signbit(b))


def test_round_to_format_binary64_is_the_correctly_rounded_conversion():
    # CPython converts a Fraction to float with one correct rounding
    # (ties to even); the definition written out must agree everywhere,
    # including ties, the subnormal range and the top binade
    rng = np.random.default_rng(23)
    cases = [Fraction(1) + Fraction(1, 2 ** 53), Fraction(1) + Fraction(3, 2 ** 53),
             Fraction(1, 2 ** 1075), Fraction(3, 2 ** 1076), Fraction(1, 2 ** 1076),
             Fraction(2 ** 53 + 1) * 2 ** 970, Fraction(1, 3), Fraction(-2, 7)]
    for _ in range(3000):
        num = int(rng.integers(1, 2 ** 62))
        den = int(rng.integers(1, 2 ** 62))
        cases.append(Fraction(num, den) * Fraction(2) ** int(rng.integers(-1130, 960)))
    for x in cases:
        assert er.round_to_format(x, er.BINARY64) == Fraction(float(x)), x


def test_round_to_format_binary32_is_ieee_single():
    # numpy's binary32 addition and division are IEEE single operations
    rng = np.random.default_rng(24)
    for _ in range(20000):
        a = np.float32(rng.standard_normal() * 2.0 ** int(rng.integers(-150, 60)))
        b = np.float32(rng.standard_normal() * 2.0 ** int(rng.integers(-150, 60)))
        got = er.add_rn(float(a), float(b), er.BINARY32)
        want = a + b
        assert np.float32(got) == want and math.copysign(1.0, got) == math.copysign(1.0, float(want))
        q = er.div_rn(float(a), 7.0, er.BINARY32)
        assert np.float32(q) == a / np.float32(7.0)
        assert math.copysign(1.0, q) == math.copysign(1.0, float(a / np.float32(7.0)))
    # a tie, and a quotient that underflows to a signed zero
    assert er.add_rn(1.0, 2.0 ** -24, er.BINARY32) == 1.0
    assert er.add_rn(1.0 + 2.0 ** -23, 2.0 ** -24, er.BINARY32) == 1.0 + 2.0 ** -22
    assert math.copysign(1.0, er.div_rn(-(2.0 ** -149), 7.0, er.BINARY32)) < 0


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 5)])
def test_seq_rule_equals_per_operation_rounding(shape):
    nx, ny, nz = shape
    u0 = rand_grid(3, nx, ny, nz)
    for k in range(1, 7):
        want = np.array(er.iterate_sequential(u0, BC_MIXED, k, er.BINARY64))
        got = oracle.jacobi(u0, BC_MIXED, k, oracle.RULE_SEQ)
        assert np.array_equal(got, want) and _signs_equal(got, want), f"iteration {k}"


def test_seq_rule_equals_per_operation_rounding_mixed_signs_and_tiny_values():
    # negative values, exact cancellations, subnormal sums and quotients that
    # underflow to a signed zero
    nx, ny, nz = 3, 4, 5
    rng = np.random.default_rng(25)
    u0 = rng.standard_normal((nz, ny, nx)) * 2.0 ** rng.integers(-40, 20, size=(nz, ny, nx))
    flat = u0.reshape(-1)
    flat[::7] = 2.0 ** -1074 * rng.integers(-5, 6, size=flat[::7].shape)
    flat[3::11] = -0.0
    flat[5::13] = -flat[4::13][: flat[5::13].size]
    bc = (-0.75, 3.0, -(2.0 ** -1073), 0.0, -0.0, 1e-300)
    for k in range(1, 5):
        want = np.array(er.iterate_sequential(u0, bc, k, er.BINARY64))
        got = oracle.jacobi(u0, bc, k, oracle.RULE_SEQ)
        assert np.array_equal(got, want) and _signs_equal(got, want), f"iteration {k}"


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 5)])
def test_f32_equals_per_operation_rounding(shape):
    nx, ny, nz = shape
    u0 = rand_grid(3, nx, ny, nz).astype(np.float32)
    bc = [float(np.float32(b)) for b in BC_MIXED]
    for k in range(1, 7):
        want = np.array(er.iterate_sequential(u0, bc, k, er.BINARY32), dtype=np.float32)
        got = oracle.jacobi_f32(u0, bc, k)
        assert np.array_equal(got, want) and _signs_equal(got, want), f"iteration {k}"


def test_f32_equals_per_operation_rounding_mixed_signs_and_tiny_values():
    nx, ny, nz = 4, 3, 4
    rng = np.random.default_rng(26)
    u0 = (rng.standard_normal((nz, ny, nx)) * 2.0 ** rng.integers(-140, 30, size=(nz, ny, nx))).astype(np.float32)
    flat = u0.reshape(-1)
    flat[::5] = np.float32(2.0 ** -149) * rng.integers(-4, 5, size=flat[::5].shape).astype(np.float32)
    flat[2::9] = np.float32(-0.0)
    bc = [float(np.float32(b)) for b in (0.5, -2.0, 2.0 ** -140, -0.0, 1e30, -1e-30)]
    for k in range(1, 5):
        want = np.array(er.iterate_sequential(u0, bc, k, er.BINARY32), dtype=np.float32)
        got = oracle.jacobi_f32(u0, bc, k)
        assert np.array_equal(got, want) and _signs_equal(got, want), f"iteration {k}"


def test_seq_and_exact_rules_differ_somewhere():
    u0 = rand_grid(5, 8, 8, 8)
    a = oracle.jacobi(u0, BC_MIXED, 3, oracle.RULE_SEQ)
    b = oracle.jacobi(u0, BC_MIXED, 3, oracle.RULE_EXACT)
    assert not np.array_equal(a, b)
    assert np.max(np.abs(a - b)) < 3 * 8 * U


def _frac_mean(vals):
    return float(sum(Fraction(v) for v in vals) / 7)


def test_exact_mean7_adversarial():
    rng = np.random.default_rng(11)
    cases = [
        [1.0, 2.0 ** -60, 0, 0, 0, 0, 0],
        [1.0, -1.0, 2.0 ** -1074, 0, 0, 0, 0],
        [2.0 ** -1074] * 7,
        [2.0 ** -1074, 0, 0, 0, 0, 0, 0],
        [3 * 2.0 ** -1074, 0, 0, 0, 0, 0, 0],
        [4 * 2.0 ** -1074, 0, 0, 0, 0, 0, 0],
        [1e300, 1e300, -1e300, 5.0, 2.0 ** -1000, -3.0, 1.0],
        [7.0, 0, 0, 0, 0, 0, 0],
        [1.0 + 2.0 ** -52, 2.0 ** -53, 0, 0, 0, 0, 0],
        [-0.5, -0.25, -0.125, 0.0, -1.0, -2.0, -4.0],
        [2.0 ** 900, 2.0 ** -900, 0, 0, 0, 0, 0],
    ]
    for _ in range(300):
        e = rng.integers(-60, 60, size=7)
        s = rng.choice([-1.0, 1.0], size=7)
        cases.append(list(s * rng.random(7) * 2.0 ** e))
    for _ in range(200):
        cases.append(list(rng.random(7)))
    for v in cases:
        assert oracle.exact_mean7(v) == _frac_mean(v), v


def test_exact_laplacian_matches_rational():
    rng = np.random.default_rng(12)
    for _ in range(300):
        c = float(rng.random() * 2.0 ** int(rng.integers(-30, 30)))
        nb = list(rng.random(6) * 2.0 ** rng.integers(-30, 30, size=6))
        want = float(sum(Fraction(x) for x in nb) - 6 * Fraction(c))
        assert oracle.exact_laplacian(c, nb) == want
    # exact cancellation gives zero
    assert oracle.exact_laplacian(0.3, [0.3] * 6) == 0.0


# ---------------------------------------------------------------- P4 dense solve
def dirichlet_solution(nx, ny, nz, bc):
    """Solve 6 u_p - sum_{interior q ~ p} u_q = sum_{ghost g ~ p} bc_g densely."""
    n = nx * ny * nz
    A = np.zeros((n, n))
    b = np.zeros(n)

    def idx(i, j, k):
        return i + nx * (j + ny * k)

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = idx(i, j, k)
                A[p, p] = 6.0
                for (ii, jj, kk, face) in ((i - 1, j, k, 0), (i + 1, j, k, 1), (i, j - 1, k, 2),
                                           (i, j + 1, k, 3), (i, j, k - 1, 4), (i, j, k + 1, 5)):
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        A[p, idx(ii, jj, kk)] -= 1.0
                    else:
                        b[p] += bc[face]
    return np.linalg.solve(A, b).reshape(nz, ny, nx)


@pytest.mark.parametrize("rule", [oracle.RULE_SEQ, oracle.RULE_EXACT])
@pytest.mark.parametrize("bc", [synth.DIRICHLET_X0, BC_MIXED, (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)])
def test_limit_is_dense_dirichlet_solution(rule, bc):
    nx, ny, nz = 4, 3, 5
    sol = dirichlet_solution(nx, ny, nz, bc)
    u0 = rand_grid(9, nx, ny, nz)
    out = oracle.jacobi(u0, bc, 400, rule)
    assert np.max(np.abs(out - sol)) < 1e-13


def test_x0_face_is_the_first_ghost_plane_along_x():
    # with 1.0 outside the x = 0 face only, the solution decreases along x and
    # is mirror-symmetric in y and z
    nx, ny, nz = 6, 5, 5
    out = oracle.jacobi(np.zeros((nz, ny, nx)), synth.DIRICHLET_X0, 600, oracle.RULE_EXACT)
    assert np.all(np.diff(out, axis=2) < 0)
    assert np.allclose(out, out[:, ::-1, :], rtol=0, atol=1e-15)
    assert np.allclose(out, out[::-1, :, :], rtol=0, atol=1e-15)


# ---------------------------------------------------------------- P5 max principle
@pytest.mark.parametrize("rule", [oracle.RULE_SEQ, oracle.RULE_EXACT])
def test_maximum_principle(rule):
    u0 = rand_grid(13, 9, 7, 8)
    for k in (1, 5, 40):
        out = oracle.jacobi(u0, synth.DIRICHLET_X0, k, rule)
        assert out.min() >= 0.0 and out.max() <= 1.0


# ---------------------------------------------------------------- P6 residual
@pytest.mark.parametrize("rule", [oracle.RULE_SEQ, oracle.RULE_EXACT])
def test_residual_monotone_and_asymptotic_rate(rule):
    nx, ny, nz = 8, 6, 7
    u = rand_grid(21, nx, ny, nz)
    rhos = [oracle.residual(u, synth.DIRICHLET_X0)]
    for _ in range(150):
        u = oracle.jacobi(u, synth.DIRICHLET_X0, 1, rule)
        rhos.append(oracle.residual(u, synth.DIRICHLET_X0))
    r = np.array(rhos)
    assert np.all(r[1:] <= r[:-1] * (1 + 1e-12))
    lam = mode_factor((nx, ny, nz), (1, 1, 1))
    assert abs(r[-1] / r[-2] - lam) < 1e-4


@pytest.mark.parametrize("n,m", [((6, 5, 7), (1, 2, 3)), ((8, 8, 8), (1, 1, 1))])
def test_residual_of_sine_mode_closed_form(n, m):
    u = sine_mode(n, m)
    mu = sum(2.0 * math.cos(math.pi * mm / (nn + 1)) - 2.0 for nn, mm in zip(n, m))
    norm = math.sqrt(math.prod((nn + 1) / 2.0 for nn in n))
    want = abs(mu) * norm
    got = oracle.residual(u, [0.0] * 6)
    assert abs(got - want) <= 1e-13 * want


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 5)])
def test_residual_matches_exact_rational(shape):
    nx, ny, nz = shape
    u = rand_grid(8, nx, ny, nz)
    want = math.sqrt(float(er.residual_sq(u, BC_MIXED)))
    got = oracle.residual(u, BC_MIXED)
    assert abs(got - want) <= 1e-14 * want


def test_residual_zero_at_fixed_point():
    assert oracle.residual(np.full((3, 3, 3), 0.7), [0.7] * 6) == 0.0


# ---------------------------------------------------------------- axis covariance
def test_axis_permutation_covariance():
    # relabelling the axes (and the boundary faces with them) relabels the
    # result; with the correctly rounded mean this holds bit for bit
    nx, ny, nz = 5, 4, 3
    u0 = rand_grid(31, nx, ny, nz)
    bc = (0.9, 0.1, 0.2, 0.3, 0.4, 0.6)
    out = oracle.jacobi(u0, bc, 6, oracle.RULE_EXACT)
    # swap x and z: array axes (z, y, x) -> (x, y, z)
    u0t = np.ascontiguousarray(np.transpose(u0, (2, 1, 0)))
    bct = (bc[4], bc[5], bc[2], bc[3], bc[0], bc[1])
    outt = oracle.jacobi(u0t, bct, 6, oracle.RULE_EXACT)
    assert np.array_equal(np.transpose(outt, (2, 1, 0)), out)
    # a y-mirror of the input mirrors the output
    bcm = (bc[0], bc[1], bc[3], bc[2], bc[4], bc[5])
    outm = oracle.jacobi(np.ascontiguousarray(u0[:, ::-1, :]), bcm, 6, oracle.RULE_EXACT)
    assert np.array_equal(outm[:, ::-1, :], out)


# ---------------------------------------------------------------- binary32
@pytest.mark.parametrize("c", [0.0, 0.5, 1.0, 3.0])
def test_f32_constant_fixed_point(c):
    u0 = np.full((4, 5, 6), c, dtype=np.float32)
    assert np.array_equal(oracle.jacobi_f32(u0, [c] * 6, 5), u0)


def test_f32_error_bound_against_f64():
    nx, ny, nz = 10, 9, 8
    u64 = rand_grid(17, nx, ny, nz)
    u32 = u64.astype(np.float32)
    k = 60
    a = oracle.jacobi(u64, synth.DIRICHLET_X0, k, oracle.RULE_EXACT)
    b = oracle.jacobi_f32(u32, synth.DIRICHLET_X0, k).astype(np.float64)
    bound = k * (27 * 2.0 ** -24 / 7 + 2.0 ** -24) + 2.0 ** -25
    err = np.max(np.abs(a - b))
    assert err <= bound
    assert err > 0


def test_f32_sine_mode():
    n, m = (6, 5, 7), (1, 2, 1)
    u0 = sine_mode(n, m).astype(np.float32)
    lam = mode_factor(n, m)
    k = 10
    out = oracle.jacobi_f32(u0, [0.0] * 6, k).astype(np.float64)
    assert np.max(np.abs(out - lam ** k * u0.astype(np.float64))) <= k * 8 * 2.0 ** -24


def test_residual_f32_uses_widened_values():
    u = rand_grid(41, 4, 4, 4).astype(np.float32)
    want = math.sqrt(float(er.residual_sq(u.astype(np.float64), [float(np.float32(b)) for b in BC_MIXED])))
    got = oracle.residual(u, BC_MIXED)
    assert abs(got - want) <= 1e-14 * want
