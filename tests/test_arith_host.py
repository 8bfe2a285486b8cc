"""The CUDA path's integer arithmetic (correctly rounded mean of seven
binary64 values, exact Laplacian term), compiled for the host, against the
oracle's wide-accumulator arithmetic and exact rationals. Covers both the
fast 128-bit-frame path and the wide fallback."""

import ctypes
import math
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_11819_gb300", "csrc")


@pytest.fixture(scope="module")
def host_lib():
    d = tempfile.mkdtemp()
    out = os.path.join(d, "libarith_host.so")
    nvcc = "nvcc" if subprocess.run(["which", "nvcc"], capture_output=True).returncode == 0 else "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "host_arith", "arith_host.cu"), "-o", out], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.host_mean7_exact.argtypes = [ctypes.c_void_p]
    lib.host_mean7_exact.restype = ctypes.c_double
    lib.host_laplacian_exact.argtypes = [ctypes.c_double, ctypes.c_void_p]
    lib.host_laplacian_exact.restype = ctypes.c_double
    lib.host_frame_mean7.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.host_frame_mean7.restype = ctypes.c_int
    lib.host_frame_laplacian.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double)]
    lib.host_frame_laplacian.restype = ctypes.c_int
    return lib


def mean_cases(rng):
    cases = [
        [1.0] * 7,
        [1.0, 0, 0, 0, 0, 0, 0],
        [0.0] * 7,
        [-0.0] * 7,
        [-0.0, 0.0, 0, 0, 0, 0, 0],
        [1.0, 2.0 ** -60, 0, 0, 0, 0, 0],
        [1.0, 2.0 ** -72, 0, 0, 0, 0, 0],
        [1.0, 2.0 ** -73, 0, 0, 0, 0, 0],
        [1.0, -1.0, 2.0 ** -1074, 0, 0, 0, 0],
        [2.0 ** -1074] * 7,
        [2.0 ** -1022] * 7,
        [2.0 ** -960] * 7,
        [2.0 ** -959, 1e-300, 0, 0, 0, 0, 0],
        [1e300] * 7,
        [-0.5, -0.25, -0.125, 0.0, -1.0, -2.0, -4.0],
        [7.0, 0, 0, 0, 0, 0, 0],
        [1.0 + 2.0 ** -52] * 7,
        [3.5 * 2.0 ** -50, 0, 0, 0, 0, 0, 0],
    ]
    for _ in range(3000):
        cases.append(list(rng.random(7)))
    for _ in range(3000):
        e = rng.integers(-80, 10, size=7)
        cases.append(list(rng.random(7) * 2.0 ** e))
    for _ in range(1000):
        e = rng.integers(-5, 5, size=7)
        s = rng.choice([-1.0, 1.0], size=7)
        cases.append(list(s * rng.random(7) * 2.0 ** e))
    for _ in range(1000):  # one sign, all negative
        cases.append(list(-rng.random(7)))
    # exact ties and near-ties at the rounding point: multiples of small units
    for _ in range(2000):
        cases.append(list(rng.integers(0, 16, size=7) * 2.0 ** -3))
    return cases


def test_mean7_exact_host_matches_oracle_and_rationals(host_lib):
    rng = np.random.default_rng(2024)
    for v in mean_cases(rng):
        a = np.ascontiguousarray(v, dtype=np.float64)
        got = host_lib.host_mean7_exact(a.ctypes.data)
        want = oracle.exact_mean7(a)
        assert np.float64(got).tobytes() == np.float64(want).tobytes(), v
    for v in mean_cases(rng)[:500]:
        a = np.ascontiguousarray(v, dtype=np.float64)
        exact = float(sum(Fraction(float(x)) for x in a) / 7)
        assert host_lib.host_mean7_exact(a.ctypes.data) == exact


def test_laplacian_exact_host_matches_oracle(host_lib):
    rng = np.random.default_rng(99)
    cases = [(0.3, [0.3] * 6), (1.0, [0.0] * 6), (0.0, [1.0] * 6), (2.0 ** -1070, [0.0] * 6),
             (1.0, [1.0, 1.0, 1.0, 1.0, 1.0, 1.0 + 2.0 ** -52]), (-1.0, [2.0] * 6)]
    for _ in range(4000):
        c = float(rng.random())
        nb = list(rng.random(6))
        cases.append((c, nb))
    for _ in range(2000):
        c = float(rng.random() * 2.0 ** int(rng.integers(-75, 3)))
        nb = list(rng.random(6) * 2.0 ** rng.integers(-75, 3, size=6))
        cases.append((c, nb))
    for _ in range(1000):  # near cancellation: neighbours average to c
        c = float(rng.random())
        nb = [c + float(x) * 2.0 ** -50 for x in rng.integers(-3, 4, size=6)]
        cases.append((c, nb))
    for c, nb in cases:
        a = np.ascontiguousarray(nb, dtype=np.float64)
        got = host_lib.host_laplacian_exact(c, a.ctypes.data)
        want = oracle.exact_laplacian(c, a)
        assert np.float64(got).tobytes() == np.float64(want).tobytes(), (c, nb)


def exp_field(x):
    return int((np.float64(x).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF))


def test_grid_frame_mean7_matches_oracle(host_lib):
    """The grid-frame fast path either declines (the kernel then takes the
    exact per-cell path) or returns exactly the correctly rounded mean."""
    rng = np.random.default_rng(7)
    fast = total = 0
    out = ctypes.c_double()
    for v in mean_cases(rng):
        a = np.ascontiguousarray(v, dtype=np.float64)
        E = max(exp_field(x) for x in a)
        # extra >= 20 puts the whole neighbourhood in the low binades of the
        # frame, where the 96-bit sum has a zero top word
        for extra in (1, 2, 5, 20, 26, 29):
            eref = max(E, 0) + extra
            total += 1
            if host_lib.host_frame_mean7(a.ctypes.data, eref, ctypes.byref(out)):
                fast += 1
                want = oracle.exact_mean7(a)
                assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), (v, eref)
    # uniform [0, 1) data must essentially always take the fast path
    ok = 0
    for _ in range(3000):
        a = np.ascontiguousarray(rng.random(7))
        ok += host_lib.host_frame_mean7(a.ctypes.data, 1024, ctypes.byref(out))
        assert out.value == oracle.exact_mean7(a)
    assert ok == 3000
    assert fast > total // 3


def test_grid_frame_laplacian_matches_oracle(host_lib):
    rng = np.random.default_rng(8)
    out = ctypes.c_double()
    cases = [(0.3, [0.3] * 6), (1.0, [0.0] * 6), (0.0, [1.0] * 6),
             (1.0, [1.0, 1.0, 1.0, 1.0, 1.0, 1.0 + 2.0 ** -52])]
    for _ in range(4000):
        cases.append((float(rng.random()), list(rng.random(6))))
    for _ in range(2000):
        c = float(rng.random())
        cases.append((c, [c + float(x) * 2.0 ** -50 for x in rng.integers(-3, 4, size=6)]))
    for _ in range(2000):
        e = rng.integers(-25, 1, size=7)
        vals = rng.random(7) * 2.0 ** e
        cases.append((float(vals[0]), list(vals[1:])))
    fast = 0
    for c, nb in cases:
        a = np.ascontiguousarray(nb, dtype=np.float64)
        eref = max(exp_field(x) for x in [c] + list(nb)) + 1
        if host_lib.host_frame_laplacian(c, a.ctypes.data, eref, ctypes.byref(out)):
            fast += 1
            want = oracle.exact_laplacian(c, a)
            assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), (c, nb)
    assert fast > 0.9 * len(cases)


def test_frame_sum7_is_the_exact_scaled_sum(host_lib):
    """The one-chain 96-bit sum equals the exact sum of the values scaled to
    frame units of 2^(eref - 1106), for values inside the 31-binade window."""
    host_lib.host_frame_sum7.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    host_lib.host_frame_sum7.restype = None
    rng = np.random.default_rng(11)
    out = np.zeros(3, dtype=np.uint32)
    for _ in range(3000):
        eref = int(rng.integers(990, 1030))
        # exponents inside [eref - 31, eref - 1], plus zeros
        e = rng.integers(eref - 31, eref, size=7)
        m = 1.0 + rng.random(7)
        v = np.array([float(np.ldexp(mi, int(ei) - 1023)) for mi, ei in zip(m, e)])
        v[rng.random(7) < 0.2] = 0.0
        host_lib.host_frame_sum7(np.ascontiguousarray(v).ctypes.data, eref, out.ctypes.data)
        got = int(out[0]) | (int(out[1]) << 32) | (int(out[2]) << 64)
        want = sum(Fraction(float(x)) * Fraction(2) ** (1106 - eref) for x in v)
        assert want.denominator == 1 and got == want.numerator, (v, eref)


def test_grid_frame_tiny_frames_decline_or_match(host_lib):
    """Frames whose window reaches the subnormal range (eref below 32), and an
    empty window (eref 1): every accepted mean is the correctly rounded one."""
    rng = np.random.default_rng(12)
    out = ctypes.c_double()
    for eref in (1, 2, 3, 17, 31, 32, 33):
        for _ in range(300):
            e = rng.integers(0, max(eref, 1), size=7)
            v = np.array([float(np.ldexp(1.0 + rng.random(), int(x) - 1023)) if x > 0
                          else float(rng.integers(0, 2 ** 20)) * 2.0 ** -1074 for x in e])
            a = np.ascontiguousarray(v)
            if host_lib.host_frame_mean7(a.ctypes.data, eref, ctypes.byref(out)):
                want = oracle.exact_mean7(a)
                assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), (list(v), eref)


def test_grid_frame_mean7_top_binades_fast_path(host_lib):
    """The fixed-shift mean for sums in the top binades of the frame equals
    the correctly rounded mean, and covers typical data."""
    host_lib.host_frame_mean7_top.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    host_lib.host_frame_mean7_top.restype = ctypes.c_int
    rng = np.random.default_rng(13)
    out = ctypes.c_double()
    hits = total = 0
    for v in mean_cases(rng):
        a = np.ascontiguousarray(v, dtype=np.float64)
        E = max(exp_field(x) for x in a)
        for extra in (1, 2, 5, 8, 20):
            eref = max(E, 0) + extra
            total += 1
            if host_lib.host_frame_mean7_top(a.ctypes.data, eref, ctypes.byref(out)):
                hits += 1
                want = oracle.exact_mean7(a)
                assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), (v, eref)
    # ties and near-ties at the rounding point with large sums
    for _ in range(3000):
        v = 0.5 + rng.integers(0, 2 ** 20, size=7) * 2.0 ** -53
        a = np.ascontiguousarray(v)
        if host_lib.host_frame_mean7_top(a.ctypes.data, 1024, ctypes.byref(out)):
            hits += 1
            assert out.value == oracle.exact_mean7(a)
    ok = 0
    for _ in range(3000):
        a = np.ascontiguousarray(rng.random(7))
        ok += host_lib.host_frame_mean7_top(a.ctypes.data, 1024, ctypes.byref(out))
    assert ok > 2900
    assert hits > total // 4



def tie_cases(rng, n, w_exp=20, eps_exp=70):
    """Triples of seven doubles around a binary64 midpoint t in [0.5, 1):
    the exact mean is t (a tie), or t plus or minus eps / 7 with eps =
    2^-eps_exp, where the bits that decide the rounding lie far below the
    53rd (with a frame whose top binade is [1, 2), eps is bit 82 - eps_exp
    of the frame sum). Values: five in [0.5, 1), one in [0.25, 0.5) and
    w = 2^-w_exp (+- eps)."""
    out = []
    w = Fraction(1, 2 ** w_exp)
    eps = Fraction(1, 2 ** eps_exp)
    while len(out) < 3 * n:
        t = Fraction(2 * int(rng.integers(2 ** 52, 2 ** 53)) + 1, 2 ** 54)  # odd multiple of 2^-54 in [0.5, 1)
        target = 7 * t - w
        v6 = Fraction(int(rng.integers(2 ** 52, 2 ** 53)), 2 ** 54)
        if ((target - v6) * 2 ** 53).denominator != 1:
            v6 += Fraction(1, 2 ** 54)
        rest = target - v6
        vs = [Fraction(int(rng.integers(2 ** 52, 2 ** 53)), 2 ** 53) for _ in range(4)]
        last = rest - sum(vs)
        if not (Fraction(1, 2) <= last < 1):
            continue
        base = [float(x) for x in vs + [last, v6]]
        for d in (0, 1, -1):
            vals = base + [float(w + d * eps)]
            assert sum(Fraction(x) for x in vals) == 7 * t + d * eps
            out.append(vals)
    return out


def test_grid_frame_mean7_ties_and_sticky_near_ties(host_lib):
    """Exact binary64 ties of the mean and near-ties decided only by bits far
    below the rounding position: both frame paths against the oracle."""
    host_lib.host_frame_mean7_top.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    host_lib.host_frame_mean7_top.restype = ctypes.c_int
    rng = np.random.default_rng(14)
    out = ctypes.c_double()
    n_top = n_gen = 0
    # the deciding bit: 12 (deep in the dropped bits), 24 (the last bit the
    # fixed-shift mean drops), 25 (the first it keeps), 1 (near the bottom)
    cases = (tie_cases(rng, 100, 20, 70) + tie_cases(rng, 100, 20, 58) + tie_cases(rng, 100, 20, 57)
             + tie_cases(rng, 100, 29, 81))
    for vals in cases:
        a = np.ascontiguousarray(vals, dtype=np.float64)
        want = oracle.exact_mean7(a)
        exact = sum(Fraction(float(x)) for x in a) / 7
        assert want == float(exact)  # the oracle's rounding of the exact mean
        assert (exact * 2 ** 53).denominator != 1  # not representable: a tie or a near-tie
        if host_lib.host_frame_mean7_top(a.ctypes.data, 1024, ctypes.byref(out)):
            n_top += 1
            assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), vals
        if host_lib.host_frame_mean7(a.ctypes.data, 1024, ctypes.byref(out)):
            n_gen += 1
            assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), vals
    assert n_top == n_gen == 1200


def test_div7d_matches_correctly_rounded_division(host_lib):
    """The integer division by 7 of the sequential rule equals IEEE division
    (correctly rounded) wherever it applies: random significands over every
    exponent, both signs, the ends of its range, and exact multiples of 7."""
    host_lib.host_div7d.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    host_lib.host_div7d.restype = ctypes.c_int
    rng = np.random.default_rng(15)
    out = ctypes.c_double()
    bits = rng.integers(0, 2 ** 63, size=200000, dtype=np.uint64) | (
        rng.integers(0, 2, size=200000, dtype=np.uint64) << np.uint64(63))
    vals = list(bits.view(np.float64))
    vals += [7.0, 3.5, 1.0, 2.0 ** -1018, 2.0 ** -1019, 2.0 ** -1020, 1.7976931348623157e308, 7.0 * 2.0 ** 1000,
             -7.0, 0.0, -0.0, 5e-324, float("inf"), float("nan")]
    vals += [float(7 * k) * 2.0 ** int(e) for k, e in zip(rng.integers(1, 2 ** 50, 2000), rng.integers(-900, 900, 2000))]
    applied = 0
    for v in vals:
        if host_lib.host_div7d(float(v), ctypes.byref(out)):
            applied += 1
            want = np.float64(v) / np.float64(7.0)
            assert np.float64(out.value).tobytes() == want.tobytes(), v
        else:
            e = (np.float64(v).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
            assert e < 4 or e == 2047, v
    assert applied > 190000


def test_dadd_nonneg_matches_ieee_addition(host_lib):
    """The integer addition of the sequential rule equals IEEE binary64
    addition (round to nearest even) wherever it applies: random pairs over
    every exponent gap (0 to 70), exact ties, carries into the next binade,
    zeros, the top of its range, and refusal (return 0) for negative,
    subnormal, infinite, NaN and too-large operands."""
    host_lib.host_dadd_nonneg.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    host_lib.host_dadd_nonneg.restype = ctypes.c_int
    rng = np.random.default_rng(17)
    out = ctypes.c_double()
    pairs = []
    n = 60000
    ea = rng.integers(1, 2045, size=n)
    gap = rng.integers(0, 71, size=n)
    eb = np.maximum(ea - gap, 1)
    ma = rng.integers(0, 2 ** 52, size=n, dtype=np.uint64)
    mb = rng.integers(0, 2 ** 52, size=n, dtype=np.uint64)
    a = ((ea.astype(np.uint64) << np.uint64(52)) | ma).view(np.float64)
    b = ((eb.astype(np.uint64) << np.uint64(52)) | mb).view(np.float64)
    pairs += list(zip(a, b)) + list(zip(b, a))
    # exact ties and near-ties: b is half an ulp of a (times an odd factor) or just off it
    for _ in range(4000):
        e = int(rng.integers(-200, 200))
        av = float(np.ldexp(1.0 + int(rng.integers(0, 2 ** 52)) * 2.0 ** -52, e))
        half = float(np.ldexp(1.0, e - 53))
        for f in (1.0, 3.0, 1.0 + 2.0 ** -40, 1.0 - 2.0 ** -40, 2.0 ** -10, 5.0):
            pairs.append((av, half * f))
    # carries into the next binade
    for e in (-1000, -3, 0, 1, 700, 1020):
        top = float(np.ldexp(2.0 - 2.0 ** -52, e))
        for bv in (np.ldexp(1.0, e - 52), np.ldexp(1.0, e - 53), np.ldexp(1.5, e - 53), np.ldexp(1.0, e)):
            pairs.append((top, float(bv)))
    pairs += [(0.0, 1.0), (1.0, 0.0), (0.0, 0.0), (1.0, 1.0), (0.5, 0.25), (1.7976931348623157e308, 1.0)]
    applied = 0
    for x, y in pairs:
        x, y = float(x), float(y)
        if host_lib.host_dadd_nonneg(x, y, ctypes.byref(out)):
            applied += 1
            want = np.float64(x) + np.float64(y)
            assert np.float64(out.value).tobytes() == want.tobytes(), (x, y)
        else:
            hi = max(x, y)
            lo = min(x, y)
            eh = int(np.float64(hi).view(np.uint64) >> np.uint64(52))
            el = int(np.float64(lo).view(np.uint64) >> np.uint64(52))
            assert not (1 <= eh <= 2044 and (1 <= el <= 2044 or lo == 0.0)), (x, y)
    assert applied > 0.95 * len(pairs)
    assert host_lib.host_dadd_nonneg(0.0, 0.0, ctypes.byref(out)) == 0  # +0 alone: the larger must be normal
    for bad in ((-1.0, 1.0), (1.0, -0.5), (5e-324, 1.0), (float("inf"), 1.0), (float("nan"), 1.0),
                (float(np.ldexp(1.0, 1022)), 1.0), (1.0, -0.0)):
        assert host_lib.host_dadd_nonneg(bad[0], bad[1], ctypes.byref(out)) == 0, bad


def test_binary32_residual_frame(host_lib):
    """The binary32 residual's 64-bit frame: values convert exactly (value =
    w * 2^(eref32 - 186)) inside the 36-binade window and are flagged outside
    it; sums of squares of 64-bit integers round once, exactly."""
    host_lib.host_of32.argtypes = [ctypes.c_float, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    host_lib.host_of32.restype = ctypes.c_int
    host_lib.host_sum_squares.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    host_lib.host_sum_squares.restype = ctypes.c_double
    rng = np.random.default_rng(16)
    w = ctypes.c_longlong()
    for _ in range(20000):
        eref32 = int(rng.integers(2, 255))
        e = int(rng.integers(max(0, eref32 - 40), eref32))
        bits = (int(rng.integers(0, 2)) << 31) | (e << 23) | int(rng.integers(0, 2 ** 23))
        v = np.array([bits], dtype=np.uint32).view(np.float32)[0]
        ok = host_lib.host_of32(float(v), eref32, ctypes.byref(w))
        inside = e != 0 and e >= eref32 - 36
        assert ok == (1 if (inside or float(v) == 0.0) else 0), (bits, eref32)
        if ok:
            assert Fraction(w.value) * Fraction(2) ** (eref32 - 186) == Fraction(float(v)), (bits, eref32)
    for _ in range(3000):
        n = int(rng.integers(1, 200))
        L = rng.integers(-(2 ** 62), 2 ** 62, size=n, dtype=np.int64)
        L[rng.random(n) < 0.3] >>= int(rng.integers(0, 60))
        scale = int(rng.integers(-400, 200))
        got = host_lib.host_sum_squares(np.ascontiguousarray(L).ctypes.data, n, scale)
        exact = sum(Fraction(int(x)) ** 2 for x in L) * Fraction(2) ** scale
        assert got == float(exact), (list(L), scale)
    for L in ([0], [1], [-1], [2 ** 62 - 1] * 200, [3, -4]):
        a = np.ascontiguousarray(L, dtype=np.int64)
        assert host_lib.host_sum_squares(a.ctypes.data, len(L), 0) == float(sum(Fraction(int(x)) ** 2 for x in L))


def test_top_quotient_multiplier_has_no_overshoot_below_2_61():
    """floor(N * ceil(2^64 / 7) / 2^64) = floor(N / 7) for every N < 2^61,
    the range of N = S >> 25 on the fixed-shift path: the multiplier's excess
    5 N / (7 2^64) stays below 1 / 7. Checked on random N, on the largest N of
    each residue class, and shown to fail further up (the bound is needed)."""
    c = (2 ** 64 + 5) // 7
    assert 7 * c == 2 ** 64 + 5
    rng = np.random.default_rng(16)
    ns = [int(x) for x in rng.integers(2 ** 57, 2 ** 61, size=20000, dtype=np.uint64)]
    ns += [2 ** 61 - 1 - k for k in range(64)] + [2 ** 57 + k for k in range(64)]
    for n in ns:
        assert (n * c) >> 64 == n // 7, n
    # above 2^64 / 5 the excess can carry past the next integer
    bad = [n for n in (2 ** 64 - 1 - k for k in range(14)) if (n * c) >> 64 != n // 7]
    assert bad


# ---------------------------------------------------------------- 64-bit frame
def _nframe_lib(host_lib):
    u64p = ctypes.POINTER(ctypes.c_ulonglong)
    host_lib.host_nframe_of.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, u64p]
    host_lib.host_nframe_of.restype = ctypes.c_int
    host_lib.host_nframe_widen.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p]
    host_lib.host_nframe_widen.restype = None
    host_lib.host_frame_of.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    host_lib.host_frame_of.restype = None
    host_lib.host_nframe_mean7.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    host_lib.host_nframe_mean7.restype = ctypes.c_int
    return host_lib


def _in_window_value(rng, eref):
    e = int(rng.integers(eref - 9, eref))
    return float(np.ldexp(1.0 + float(rng.integers(0, 2 ** 52)) * 2.0 ** -52, e - 1023))


def test_narrow_frame_conversion_is_the_exact_scaled_value(host_lib):
    """A value is accepted exactly when it is a positive normal number whose
    exponent field lies in [eref - 9, eref - 1] (or +0 in the zero-accepting
    form), and its frame integer is then v * 2^(1084 - eref) exactly; widened,
    it equals the 96-bit frame value of the same number."""
    lib = _nframe_lib(host_lib)
    rng = np.random.default_rng(31)
    w = ctypes.c_ulonglong()
    wide = np.zeros(4, dtype=np.uint32)
    widened = np.zeros(3, dtype=np.uint32)
    for _ in range(6000):
        eref = int(rng.integers(13, 2048))
        kind = int(rng.integers(0, 6))
        if kind <= 2:
            v = _in_window_value(rng, eref)
        elif kind == 3:  # just outside, below or above
            e = eref - 10 if rng.random() < 0.5 else eref
            v = float(np.ldexp(1.0 + rng.random(), min(max(e, 1), 2046) - 1023))
        elif kind == 4:
            v = -_in_window_value(rng, eref)
        else:
            v = [0.0, -0.0, 2.0 ** -1074, 2.0 ** -1030 * 3][int(rng.integers(0, 4))]
        fe = exp_field(v)
        inside = v > 0 and eref - 9 <= fe <= eref - 1
        for zero_ok in (0, 1):
            ok = lib.host_nframe_of(v, eref, zero_ok, ctypes.byref(w))
            want_ok = inside or (zero_ok == 1 and v == 0.0 and math.copysign(1.0, v) > 0)
            assert bool(ok) == want_ok, (v, eref, zero_ok)
            if ok:
                exact = Fraction(v) * Fraction(2) ** (1084 - eref)
                assert exact.denominator == 1 and w.value == exact.numerator, (v, eref)
                if v != 0.0:
                    lib.host_frame_of(v, eref, wide.ctypes.data)
                    lib.host_nframe_widen(w.value, widened.ctypes.data)
                    assert list(widened) == list(wide[:3]), (v, eref)


def test_narrow_frame_mean7_matches_oracle(host_lib):
    """Wherever the 64-bit frame accepts a cell and its neighbours, its mean
    is the correctly rounded one: random data over the whole window (sums
    from 2^52 to 7 * 2^61, so every normalising shift), zeros among the
    neighbours, the largest and smallest values, and typical [0, 1) data
    (which it must essentially always accept)."""
    lib = _nframe_lib(host_lib)
    rng = np.random.default_rng(32)
    out = ctypes.c_double()
    hits = 0
    cases = []
    for _ in range(20000):
        eref = int(rng.integers(13, 2048))
        v = [_in_window_value(rng, eref) for _ in range(7)]
        for i in range(1, 7):
            if rng.random() < 0.15:
                v[i] = 0.0
        cases.append((v, eref))
    for eref in (13, 14, 1024, 2047):
        lo = float(np.ldexp(1.0, eref - 9 - 1023))
        hi = float(np.ldexp(2.0 - 2.0 ** -52, eref - 1 - 1023))
        cases += [([lo] + [0.0] * 6, eref), ([lo] * 7, eref), ([hi] * 7, eref), ([hi] + [lo] * 6, eref),
                  ([lo] + [hi] * 6, eref), ([hi] + [0.0] * 6, eref)]
    for v, eref in cases:
        a = np.ascontiguousarray(v, dtype=np.float64)
        assert lib.host_nframe_mean7(a.ctypes.data, eref, ctypes.byref(out)), (v, eref)
        want = oracle.exact_mean7(a)
        assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), (v, eref)
        hits += 1
    ok = 0
    for _ in range(5000):
        a = np.ascontiguousarray(rng.random(7))
        if lib.host_nframe_mean7(a.ctypes.data, 1024, ctypes.byref(out)):
            ok += 1
            assert out.value == oracle.exact_mean7(a)
    assert ok > 4700
    # the general cases: accepted only inside the window, and then exact
    for v in mean_cases(rng):
        a = np.ascontiguousarray(v, dtype=np.float64)
        E = max(exp_field(x) for x in a)
        for extra in (1, 2, 5, 9):
            eref = max(E, 0) + extra
            if lib.host_nframe_mean7(a.ctypes.data, eref, ctypes.byref(out)):
                want = oracle.exact_mean7(a)
                assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), (v, eref)


def narrow_tie_cases(rng, n):
    """Seven values in [2^-8, 1) whose exact sum is 7t + d 2^-60, t an odd
    multiple of 2^-54 in [0.5, 1) (a binary64 midpoint) and d in
    {0, 1, -1, 8, -8}: exact ties of the mean, and near-ties decided by the
    last unit of the 64-bit frame (2^-60 for a frame whose top binade is
    [1, 2)). With d = +-8 the three bits the normalised sum drops are zero, so
    only the remainder of the division tells a near-tie from a tie."""
    out = []
    u = Fraction(1, 2 ** 60)
    while len(out) < 5 * n:
        t = Fraction(2 * int(rng.integers(2 ** 52, 2 ** 53)) + 1, 2 ** 54)
        w = Fraction(int(rng.integers(2 ** 46, 2 ** 47)), 2 ** 54)  # in [2^-8, 2^-7)
        a4 = [Fraction(int(rng.integers(2 ** 52, 2 ** 53)), 2 ** 53) for _ in range(4)]
        R = 7 * t - w - sum(a4)
        lo = max(Fraction(1, 2), R - Fraction(1, 2))
        hi = min(Fraction(1), R - Fraction(1, 4))
        if lo >= hi:
            continue
        a5 = Fraction(int(rng.integers(math.ceil(lo * 2 ** 53), math.floor(hi * 2 ** 53))), 2 ** 53)
        a6 = R - a5
        if not (Fraction(1, 4) <= a6 < Fraction(1, 2)) or (a6 * 2 ** 54).denominator != 1:
            continue
        for d in (0, 1, -1, 8, -8):
            vals = [float(x) for x in a4 + [a5, a6, w + d * u]]
            assert sum(Fraction(x) for x in vals) == 7 * t + d * u
            out.append(vals)
    return out


def test_narrow_frame_mean7_ties_and_near_ties(host_lib):
    lib = _nframe_lib(host_lib)
    rng = np.random.default_rng(33)
    out = ctypes.c_double()
    n = 0
    for vals in narrow_tie_cases(rng, 400):
        a = np.ascontiguousarray(vals, dtype=np.float64)
        exact = sum(Fraction(float(x)) for x in a) / 7
        assert (exact * 2 ** 53).denominator != 1  # not representable: a tie or a near-tie
        want = oracle.exact_mean7(a)
        assert want == float(exact)
        for order in (a, a[::-1].copy()):
            assert lib.host_nframe_mean7(order.ctypes.data, 1024, ctypes.byref(out))
            assert np.float64(out.value).tobytes() == np.float64(want).tobytes(), vals
            n += 1
    assert n == 4000


# ---- binary32 residual in split words (the update launch's residual term)

def _r32_bind(lib):
    lib.host_r32_split.argtypes = [ctypes.c_float, ctypes.c_int, ctypes.c_void_p]
    lib.host_r32_split.restype = ctypes.c_int
    lib.host_r32_laplacian.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.host_r32_laplacian.restype = ctypes.c_int
    lib.host_r32_sum_squares.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]
    lib.host_r32_sum_squares.restype = ctypes.c_int
    lib.host_r32_combine.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.host_r32_combine.restype = None
    return lib


def _f32_cases(rng, f, n):
    """binary32 values below 2^(E - 1) (E = f - 125): random magnitudes over
    40 binades below the top, zeros, the extremes and the split's boundaries."""
    E = f - 125
    top = np.nextafter(np.float32(2.0 ** (E - 1)), np.float32(0))
    q1 = 2.0 ** (E - 22)
    special = [0.0, -0.0, top, -top, q1, -q1, q1 / 2, 1.5 * q1, 2.5 * q1, np.nextafter(np.float32(q1), np.float32(0)),
               2.0 ** (E - 45), 3 * 2.0 ** (E - 45), 2.0 ** (E - 46), 2.0 ** (E - 23) * 1.25]
    e = rng.uniform(E - 41, E - 1, n)
    v = (2.0 ** e) * rng.choice([-1.0, 1.0], n)
    out = np.concatenate([np.array(special, dtype=np.float64), v]).astype(np.float32)
    return out[np.abs(out.astype(np.float64)) < 2.0 ** (E - 1)]


@pytest.mark.parametrize("f", [127, 150, 40, 230])
def test_r32_split_is_exact_exactly_where_it_reports_so(host_lib, f):
    lib = _r32_bind(host_lib)
    E = f - 125
    q1, q2 = Fraction(2) ** (E - 22), Fraction(2) ** (E - 45)
    hg = (ctypes.c_int32 * 2)()
    n_exact = n_inexact = 0
    for v in _f32_cases(np.random.default_rng(f), f, 3000):
        rc = lib.host_r32_split(float(v), f, hg)
        fv = Fraction(float(v))
        exact = (fv / q2).denominator == 1
        assert rc == (1 if exact else 0), (v, rc)
        if abs(fv) >= q1:
            assert rc == 1, v  # the window: every value within 21 binades of the top
        if rc == 1:
            n_exact += 1
            assert hg[0] * q1 + hg[1] * q2 == fv, v
            assert abs(hg[0]) <= 2 ** 21 and abs(hg[1]) <= 2 ** 22
        else:
            n_inexact += 1
    assert n_exact > 1000 and n_inexact > 100


def test_r32_split_declines_frames_out_of_range(host_lib):
    lib = _r32_bind(host_lib)
    hg = (ctypes.c_int32 * 2)()
    assert lib.host_r32_split(1.0, 251, hg) == -1  # E = 126: C1 = 1.5 * 2^127 would overflow
    assert lib.host_r32_split(0.0, 24, hg) == -1  # E = -101: C2 would be subnormal
    assert lib.host_r32_split(1.0, 250, hg) != -1 and lib.host_r32_split(0.0, 25, hg) != -1


@pytest.mark.parametrize("f", [127, 100])
def test_r32_laplacian_parts_are_the_exact_term(host_lib, f):
    lib = _r32_bind(host_lib)
    E = f - 125
    q2 = Fraction(2) ** (E - 45)
    rng = np.random.default_rng(7 + f)
    top = np.nextafter(np.float32(2.0 ** (E - 1)), np.float32(0))
    lhg = (ctypes.c_int32 * 2)()
    cases = [np.array([-top] + [top] * 6, dtype=np.float32), np.array([top] + [-top] * 6, dtype=np.float32),
             np.zeros(7, dtype=np.float32), np.array([top] * 7, dtype=np.float32)]
    for _ in range(3000):
        e = rng.uniform(E - 22, E - 1, 7)
        s = rng.choice([-1.0, 1.0], 7) if rng.random() < 0.5 else np.ones(7)
        v = (2.0 ** e * s).astype(np.float32)
        v[rng.random(7) < 0.1] = 0.0
        cases.append(v)
    for v in cases:
        v = np.ascontiguousarray(v, dtype=np.float32)
        assert lib.host_r32_laplacian(v.ctypes.data, f, lhg) == 1
        fr = [Fraction(float(x)) for x in v]
        L = sum(fr[1:]) - 6 * fr[0]
        assert (lhg[0] * 2 ** 23 + lhg[1]) * q2 == L, v
        assert abs(lhg[0]) <= 12 * 2 ** 21 and abs(lhg[1]) <= 12 * 2 ** 22


def test_r32_sum_of_squares_is_exact_then_rounded_once(host_lib):
    lib = _r32_bind(host_lib)
    f = 127
    E = f - 125
    q2 = Fraction(2) ** (E - 45)
    rng = np.random.default_rng(11)
    top = np.nextafter(np.float32(2.0 ** (E - 1)), np.float32(0))
    # 2048 cells (the most one thread sums): extreme terms, near-cancelling
    # ones and random ones
    n = 2048
    v = (2.0 ** rng.uniform(E - 22, E - 1, (n, 7)) * rng.choice([-1.0, 1.0], (n, 7))).astype(np.float32)
    v[:512, 0] = -top
    v[:512, 1:] = top
    v[512:1024, 1:] = v[512:1024, :1]  # L = 0
    v[1024:1100, 1] = np.nextafter(v[1024:1100, 1], np.float32(0))  # L = one spacing
    v = np.ascontiguousarray(v)
    acc3 = (ctypes.c_int64 * 3)()
    out = ctypes.c_double()
    assert lib.host_r32_sum_squares(v.ctypes.data, n, f, acc3, ctypes.byref(out)) == 1
    exact = Fraction(0)
    for row in v:
        fr = [Fraction(float(x)) for x in row]
        exact += (sum(fr[1:]) - 6 * fr[0]) ** 2
    assert out.value == float(exact)
    assert (acc3[0] * 2 ** 46 + acc3[1] * 2 ** 24 + acc3[2]) * q2 * q2 == exact
    assert max(abs(acc3[0]), abs(acc3[1]), abs(acc3[2])) < 2 ** 63
    # a value outside the window makes the sum report itself inexact
    v[5, 3] = np.float32(2.0 ** (E - 30) * 1.3)
    assert lib.host_r32_sum_squares(v.ctypes.data, n, f, acc3, ctypes.byref(out)) == 0


def test_r32_combine_is_the_128_bit_sum(host_lib):
    lib = _r32_bind(host_lib)
    rng = np.random.default_rng(3)
    abc = (ctypes.c_int64 * 3)()
    lohi = (ctypes.c_uint64 * 2)()
    for _ in range(2000):
        vals = [int(rng.integers(-2 ** 62, 2 ** 62)) for _ in range(3)]
        if rng.random() < 0.3:
            vals[int(rng.integers(0, 3))] = int(rng.choice([2 ** 63 - 1, -2 ** 63, 0, -1]))
        abc[0], abc[1], abc[2] = vals
        lib.host_r32_combine(abc, lohi)
        s = (vals[0] * 2 ** 46 + vals[1] * 2 ** 24 + vals[2]) % 2 ** 128
        assert lohi[0] + 2 ** 64 * lohi[1] == s, vals


def test_nframe_residual_is_the_exact_sum_of_squares_rounded_once(host_lib):
    """The binary64 residual of the 64-bit frame: L = S - 7c of the frame
    integers is the exact Laplacian term, and the 192-bit sum of squares over
    512 cells (the most one thread sums) is rounded once."""
    lib = host_lib
    lib.host_nframe_residual.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.host_nframe_residual.restype = ctypes.c_int
    rng = np.random.default_rng(17)
    out = ctypes.c_double()
    for eref in (1024, 1030, 600, 1500):
        # the window: exponent fields eref - 9 .. eref - 1, values in [2^(eref-1032), 2^(eref-1023))
        top = 2.0 ** (eref - 1023) * (1 - 2.0 ** -53)
        low = 2.0 ** (eref - 1032)
        n = 512
        v = low * 2.0 ** rng.uniform(0, 8.99, (n, 7))
        v[:64, 0] = low
        v[:64, 1:] = top  # L near its largest, 6 * 2^61 frame units
        v[64:128, 0] = top
        v[64:128, 1:] = low  # L near its most negative
        v[128:192, 1:] = v[128:192, :1]  # L = 0
        v[200:260, 3] = 0.0  # zero neighbours are in the frame
        v = np.ascontiguousarray(v)
        assert lib.host_nframe_residual(v.ctypes.data, n, eref, ctypes.byref(out)) == 1
        exact = Fraction(0)
        for row in v:
            fr = [Fraction(float(x)) for x in row]
            exact += (sum(fr[1:]) - 6 * fr[0]) ** 2
        assert out.value == float(exact), eref
    # a value below the window, or a zero centre, is reported
    w = np.ascontiguousarray(np.full((1, 7), 0.75))
    w[0, 2] = 2.0 ** -20
    assert lib.host_nframe_residual(w.ctypes.data, 1, 1024, ctypes.byref(out)) == 0
    w[0, 2] = 0.75
    w[0, 0] = 0.0
    assert lib.host_nframe_residual(w.ctypes.data, 1, 1024, ctypes.byref(out)) == 0
