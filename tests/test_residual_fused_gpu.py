"""The residual inside the update launch (jac_iterate_residual) and the
residual launch that shares its arithmetic, binary32 and binary64, against
the oracle.

- The grid after the iterations: bit-exact against the oracle (binary32; the
  correctly rounded mean or the left-to-right rule for binary64).
- rho(u^k): within 1e-12 relative of oracle.residual of the oracle's u^k
  (both are the exact sum of L^2 rounded once, then the per-unit partials
  summed in binary64: a few units of 2^-53 apart).
- rho(u^k) has the same bits as jac_residual on the same grid in the same
  configuration (one per-unit arithmetic, one summation order).
Cases: several blocks with ragged tiles, blocks of odd x extent (the
two-plane fallback engine), values outside the exact range, frames out of
it, mixed signs.
"""

import numpy as np
import pytest

import oracle
import synth
from paper_2202_11819_gb300 import Jacobi3D, _lib

pytestmark = pytest.mark.gpu

FUSED = ["fused", "graph_fused"]
OTHER = ["persistent", "unfused"]
BC_MIXED = (1.0, 0.25, 0.0, 0.5, 0.125, 0.75)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.load()
    yield


def ctx(dims, block, bc, mode, dtype, arith):
    return Jacobi3D(dims, block, dtype=dtype, bc=bc, mode=mode, arith=arith if dtype == "f64" else "seq")


def iterate_residual(u0, dims, block, n, every, mode, bc, dtype="f32", arith="exact"):
    import torch

    with ctx(dims, block, bc, mode, dtype, arith) as J:
        J.write(u0)
        out = torch.full((max(1, -(-n // every)),), float("nan"), dtype=torch.float64, device="cuda")
        J.iterate_residual(n, every, out)
        J.sync()
        return J.read(np.float32 if dtype == "f32" else np.float64), out.cpu().numpy()


def standalone_residuals(u0, dims, block, n, every, mode, bc, dtype="f32", arith="exact"):
    rhos = []
    with ctx(dims, block, bc, mode, dtype, arith) as J:
        J.write(u0)
        for k in range(0, n, every):
            if k:
                J.iterate(every)
            rhos.append(J.residual())
    return np.array(rhos)


def oracle_iterate(u, bc, n, dtype, arith):
    if dtype == "f32":
        return oracle.jacobi_f32(u, bc, n)
    return oracle.jacobi(u, bc, n, oracle.RULE_EXACT if arith == "exact" else oracle.RULE_SEQ)


def check(u0, dims, block, n, every, mode, bc, dtype="f32", arith="exact"):
    got, rho = iterate_residual(u0, dims, block, n, every, mode, bc, dtype, arith)
    assert np.array_equal(got, oracle_iterate(u0, bc, n, dtype, arith))
    ks = list(range(0, n, every))
    assert len(rho) == len(ks)
    uk = u0
    for j, k in enumerate(ks):
        if k:
            uk = oracle_iterate(uk, bc, every, dtype, arith)
        want = oracle.residual(uk, bc)
        assert abs(rho[j] - want) <= 1e-12 * want, (j, k, rho[j], want)
    assert np.array_equal(rho, standalone_residuals(u0, dims, block, n, every, mode, bc, dtype, arith))
    return rho


CASES = [
    ((40, 24, 20), (16, 8, 10)),    # tiles overhanging every block edge
    ((70, 33, 21), (34, 17, 11)),   # uneven split, ragged y
    ((45, 20, 12), (15, 10, 6)),    # odd x extent: the fallback engine for every unit
    ((130, 9, 7), (130, 9, 7)),     # one block: 64 + 64 + 2 wide tiles
]


@pytest.mark.parametrize("mode", FUSED + OTHER)
@pytest.mark.parametrize("dims,block", CASES)
def test_iterate_residual_matches_oracle_and_standalone(dims, block, mode):
    u0 = synth.grid_uniform01(31, *dims).astype(np.float32)
    check(u0, dims, block, 11, 4, mode, BC_MIXED)  # rho of u^0, u^4, u^8


@pytest.mark.parametrize("arith", ["exact", "seq"])
@pytest.mark.parametrize("mode", FUSED + OTHER)
@pytest.mark.parametrize("dims,block", CASES)
def test_iterate_residual_binary64(dims, block, mode, arith):
    u0 = synth.grid_uniform01(37, *dims)
    check(u0, dims, block, 11, 4, mode, BC_MIXED, "f64", arith)


@pytest.mark.parametrize("mode", FUSED)
@pytest.mark.parametrize("case", ["spread", "mixed_signs", "huge_frame", "tiny_frame", "zeros"])
def test_iterate_residual_binary64_outside_the_frame(mode, case):
    """Binary64 units whose steps take the 96-bit frame (values more than
    nine binades apart, negative values), and grids whose sum of squares the
    integer form could not scale, go to the two-plane engine."""
    dims, block = (48, 20, 14), (24, 10, 7)
    rng = np.random.default_rng(8)
    u0 = rng.random(dims[::-1]) + 0.5
    bc = BC_MIXED
    if case == "spread":
        u0.reshape(-1)[::89] = 3e-7
    elif case == "mixed_signs":
        u0 = u0 - 1.0
        bc = (1.0, -0.25, 0.0, 0.5, -0.125, 0.75)
    elif case == "huge_frame":  # squares scaled by 2^810: beyond the integer form's range, finite in binary64
        u0 = u0 * 1e140
        bc = tuple(b * 1e140 for b in BC_MIXED)
    elif case == "tiny_frame":  # squares scaled by 2^-1050
        u0 = u0 * 1e-140
        bc = tuple(b * 1e-140 for b in BC_MIXED)
    else:
        u0.reshape(-1)[::3] = 0.0
        bc = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)
    check(u0, dims, block, 5, 2, mode, bc, "f64", "exact")


@pytest.mark.parametrize("mode", FUSED)
@pytest.mark.parametrize("case", ["tiny", "mixed_signs", "huge_frame", "minute_frame", "zeros"])
def test_iterate_residual_outside_the_split(mode, case):
    """Units with a value more than 21 binades below the grid's largest, and
    grids whose frame the split's constants cannot take, go to the fallback
    engine; mixed signs and zeros stay on the split."""
    dims, block = (48, 20, 14), (24, 10, 7)
    rng = np.random.default_rng(5)
    u0 = rng.random(dims[::-1]).astype(np.float32)
    bc = BC_MIXED
    if case == "tiny":
        u0.reshape(-1)[::97] = np.float32(3e-9)
    elif case == "mixed_signs":
        u0 = (u0 - np.float32(0.5)).astype(np.float32)
        bc = (1.0, -0.25, 0.0, 0.5, -0.125, 0.75)
    elif case == "huge_frame":  # largest exponent field 252: C1 would overflow
        u0 = ((u0 + np.float32(1.0)) * np.float32(2.2e37)).astype(np.float32)
        bc = tuple(float(np.float32(b * 2.2e37)) for b in BC_MIXED)
    elif case == "minute_frame":  # largest exponent field 20: C2 would be subnormal
        u0 = ((u0 + np.float32(1.0)) * np.float32(1e-32)).astype(np.float32)
        bc = tuple(float(np.float32(b * 1e-32)) for b in BC_MIXED)
    else:
        u0.reshape(-1)[::3] = 0.0
        bc = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)
    check(u0, dims, block, 5, 2, mode, bc)


def test_iterate_residual_counts_and_errors():
    import torch

    dims, block = (32, 16, 12), (16, 8, 6)
    u0 = synth.grid_uniform01(2, *dims).astype(np.float32)
    with Jacobi3D(dims, block, dtype="f32", bc=BC_MIXED, mode="fused") as J:
        J.write(u0)
        out = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
        J.iterate_residual(0, 3, out)  # nothing enqueued, nothing written
        J.iterate_residual(7, 1, out)  # every iteration: 7 residuals
        J.sync()
        o = out.cpu().numpy()
        assert np.all(o[:7] > 0) and o[7] == -1.0
        assert J.info()["iterations"] == 7
        with pytest.raises(_lib.JacError) as e:
            _lib.jac_iterate_residual(J.h, 3, 0, out.data_ptr())
        assert e.value.code == _lib.JAC_EINVAL
        with pytest.raises(_lib.JacError) as e:
            _lib.jac_iterate_residual(J.h, 3, 1, 0)
        assert e.value.code == _lib.JAC_EINVAL
        with pytest.raises(ValueError):
            J.iterate_residual(7, 2, out[:3])
        with pytest.raises(ValueError):
            J.iterate_residual(7, 2, torch.zeros(8, dtype=torch.float32, device="cuda"))
        with pytest.raises(ValueError):
            J.iterate_residual(7, 2, torch.zeros(8, dtype=torch.float64))
        assert np.array_equal(J.read(np.float32), oracle.jacobi_f32(u0, BC_MIXED, 7))


def test_fused_residual_at_full_size_equals_the_residual_launch():
    """1024^3 binary32 in 64^3 blocks with the tile the autotuner picks there
    (64 wide): the residual from the update launch has the residual launch's
    bits, and the iteration the update launch's."""
    import torch

    dims, block = (1024, 1024, 1024), (64, 64, 64)
    u0 = torch.from_numpy(synth.grid_uniform01(0, *dims).reshape(-1)).to("cuda").to(torch.float32)
    with Jacobi3D(dims, block, dtype="f32", bc=synth.DIRICHLET_X0, mode="fused") as J:
        _lib.jac_set_tile(J.h, 64, 0)
        J.write_device(u0)
        J.iterate(60)  # an aged field, as the bench's residuals see it
        rho = torch.zeros(2, dtype=torch.float64, device="cuda")
        J.residual_device(rho[0:1])
        J.iterate_residual(1, 1, rho[1:2])
        a = torch.empty_like(u0)
        J.read_device(a)
        J.write_device(u0)
        J.iterate(61)
        b = torch.empty_like(u0)
        J.read_device(b)
        J.sync()
    r = rho.cpu().numpy()
    assert r[0] == r[1] and r[0] > 0
    assert torch.equal(a, b)


def test_binary64_fused_residual_at_full_size_equals_the_residual_launch():
    """512^3 binary64 in 64^3 blocks, 64-wide tiles, the correctly rounded
    mean in the fused form: the residual from the update launch has the
    residual launch's bits, and the iteration the plain fused launch's."""
    import torch

    dims, block = (512, 512, 512), (64, 64, 64)
    u0 = torch.from_numpy(synth.grid_uniform01(0, *dims).reshape(-1)).to("cuda")
    with Jacobi3D(dims, block, bc=synth.DIRICHLET_X0, mode="fused", arith="exact") as J:
        _lib.jac_set_tile(J.h, 64, 0)
        J.write_device(u0)
        J.iterate(60)
        rho = torch.zeros(2, dtype=torch.float64, device="cuda")
        J.residual_device(rho[0:1])
        J.iterate_residual(1, 1, rho[1:2])
        a = torch.empty_like(u0)
        J.read_device(a)
        J.write_device(u0)
        J.iterate(61)
        b = torch.empty_like(u0)
        J.read_device(b)
        J.sync()
    r = rho.cpu().numpy()
    assert r[0] == r[1] and r[0] > 0
    assert torch.equal(a, b)


@pytest.mark.parametrize("mode", FUSED + ["persistent"])
def test_binary64_residual_at_the_frame_extremes(mode):
    """A checkerboard of 1.9 and 0.004 (both inside one nine-binade window of
    the 64-bit frame): every cell's Laplacian term is about six times the
    window's top in magnitude, beyond 2^63 frame units, so the integer form
    must square its magnitude unsigned."""
    dims, block = (48, 20, 14), (24, 10, 7)
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    u0 = np.where((x + y + z) % 2 == 0, 1.9, 0.004)
    bc = (1.0, 0.5, 0.25, 1.5, 0.75, 1.25)
    check(u0, dims, block, 3, 1, mode, bc, "f64", "exact")
