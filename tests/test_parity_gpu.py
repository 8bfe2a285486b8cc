"""GPU parity: libjacobi3d (through the C ABI) against the CPU oracle.

Tolerances:
- binary64 with JAC_ARITH_SEQ against the oracle's left-to-right rule and
  JAC_ARITH_EXACT against the oracle's correctly rounded mean: bit-exact;
- JAC_ARITH_EXACT against the left-to-right oracle: |diff| <= 1e-12 * max|u|
  (per iteration the two roundings differ by at most 2.43 + 0.5 units of
  2^-52 * max|u|, and the averaging operator does not expand max-norm
  differences, so n iterations differ by at most n * 6.5e-16 * max|u|);
- binary32 against the binary32 oracle: bit-exact;
- residual: 1e-12 relative.
"""

import numpy as np
import pytest

import oracle
import synth
from paper_2202_11819_gb300 import Jacobi3D, _lib

pytestmark = pytest.mark.gpu

MODES = ["unfused", "fused", "graph", "persistent", "graph_fused", "split"]
BC_MIXED = (1.0, 0.25, 0.0, 0.5, 0.125, 0.75)
ORACLE_RULE = {"seq": oracle.RULE_SEQ, "exact": oracle.RULE_EXACT}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.load()
    yield


def run(u0, dims, block, iters, mode, arith="exact", bc=synth.DIRICHLET_X0, dtype="f64", chunks=None):
    with Jacobi3D(dims, block, dtype=dtype, bc=bc, mode=mode, arith=arith if dtype == "f64" else "seq") as J:
        J.write(u0)
        for n in (chunks or [iters]):
            J.iterate(n)
        out = J.read(np.float32 if dtype == "f32" else np.float64)
        rho = J.residual()
    return out, rho


def grid(seed, dims):
    return synth.grid_uniform01(seed, *dims).copy()


@pytest.mark.parametrize("arith", ["seq", "exact"])
@pytest.mark.parametrize("mode", MODES)
def test_plain_64cubed_one_block_100_iterations(mode, arith):
    dims = (64, 64, 64)
    u0 = grid(0, dims)
    want = oracle.jacobi(u0, synth.DIRICHLET_X0, 100, ORACLE_RULE[arith])
    got, _ = run(u0, dims, dims, 100, mode, arith)
    assert np.array_equal(got, want)


CASES = [
    ((16, 16, 16), (8, 8, 8)),
    ((20, 13, 7), (8, 5, 3)),
    ((200, 40, 30), (100, 17, 16)),  # two x tiles per block with a ragged tail; uneven y/z split
    ((300, 5, 6), (256, 5, 6)),       # blocks of 150 in x: three tiles of 64, 64, 22
    ((1, 1, 1), (1, 1, 1)),
    ((9, 1, 4), (2, 1, 1)),
]


@pytest.mark.parametrize("arith", ["seq", "exact"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dims,block", CASES)
def test_overdecomposed_grids_bit_exact(dims, block, mode, arith):
    u0 = grid(3, dims)
    iters = 7  # odd: ends on the other buffer
    want = oracle.jacobi(u0, BC_MIXED, iters, ORACLE_RULE[arith])
    got, _ = run(u0, dims, block, iters, mode, arith, bc=BC_MIXED)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", MODES)
def test_iterations_split_across_calls_and_modes(mode):
    dims, block = (24, 18, 10), (8, 6, 5)
    u0 = grid(5, dims)
    want = oracle.jacobi(u0, BC_MIXED, 9, oracle.RULE_EXACT)
    with Jacobi3D(dims, block, bc=BC_MIXED, mode=mode) as J:
        J.write(u0)
        J.iterate(2)
        J.set_mode("persistent")
        J.iterate(3)
        J.set_mode("unfused")
        J.iterate(1)
        J.set_mode(mode)
        J.iterate(3)
        got = J.read()
    assert np.array_equal(got, want)


def test_decomposition_independence():
    dims = (40, 36, 28)
    u0 = grid(7, dims)
    outs = []
    for block in [(40, 36, 28), (20, 18, 14), (13, 7, 9), (64 if dims[0] >= 64 else 40, 5, 3), (1, 36, 28)]:
        got, _ = run(u0, dims, block, 11, "persistent", "exact", bc=BC_MIXED)
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("mode", ["unfused", "fused", "persistent", "graph"])
def test_f32_bit_exact(mode):
    dims, block = (40, 24, 20), (16, 8, 10)
    u0 = grid(9, dims).astype(np.float32)
    want = oracle.jacobi_f32(u0, BC_MIXED, 13)
    got, _ = run(u0, dims, block, 13, mode, bc=BC_MIXED, dtype="f32")
    assert np.array_equal(got, want)


def test_exact_arith_within_bound_of_sequential_oracle():
    dims, block = (48, 40, 32), (16, 16, 16)
    u0 = grid(11, dims)
    n = 60
    want = oracle.jacobi(u0, synth.DIRICHLET_X0, n, oracle.RULE_SEQ)
    got, _ = run(u0, dims, block, n, "persistent", "exact")
    assert np.max(np.abs(got - want)) <= min(1e-12, n * 6.5e-16) * 1.0


def test_exact_arith_slow_paths():
    # negative values, mixed signs, subnormals, exact zeros and wide exponent
    # spreads force the wide-accumulator path of the correctly rounded mean
    dims, block = (18, 10, 9), (6, 5, 3)
    rng = np.random.default_rng(1)
    u0 = rng.random(dims[::-1]) * 2.0 ** rng.integers(-80, 40, size=dims[::-1])
    u0 *= rng.choice([-1.0, 1.0], size=u0.shape)
    u0.reshape(-1)[::17] = 0.0
    u0.reshape(-1)[5::23] = 2.0 ** -1070
    u0.reshape(-1)[7::29] = -(2.0 ** -1050)
    bc = (3.0, -2.0, 1e-200, 0.0, -5e10, 7.0)
    want = oracle.jacobi(u0, bc, 5, oracle.RULE_EXACT)
    got, _ = run(u0, dims, block, 5, "fused", "exact", bc=bc)
    assert np.array_equal(got, want)
    got2, _ = run(u0, dims, block, 5, "persistent", "exact", bc=bc)
    assert np.array_equal(got2, want)


@pytest.mark.parametrize("mode", MODES)
def test_sequential_rule_special_values(mode):
    """The sequential rule on values its integer first addition and integer
    division refuse (negative, subnormal, zero, sums whose quotient leaves the
    normal range): those lanes take the binary64 pipe, and every cell stays
    bit-exact against the oracle."""
    dims, block = (18, 10, 9), (6, 5, 3)
    rng = np.random.default_rng(2)
    u0 = rng.random(dims[::-1]) * 2.0 ** rng.integers(-80, 40, size=dims[::-1])
    u0 *= rng.choice([-1.0, 1.0], size=u0.shape)
    u0.reshape(-1)[::17] = 0.0
    u0.reshape(-1)[5::23] = 2.0 ** -1070
    u0.reshape(-1)[7::29] = -(2.0 ** -1050)
    u0.reshape(-1)[3::31] = 2.0 ** -1020
    bc = (3.0, -2.0, 1e-200, 0.0, -5e10, 7.0)
    want = oracle.jacobi(u0, bc, 5, oracle.RULE_SEQ)
    got, _ = run(u0, dims, block, 5, mode, "seq", bc=bc)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_residual_parity(dtype):
    dims, block = (30, 22, 18), (10, 11, 6)
    u0 = grid(13, dims)
    if dtype == "f32":
        u0 = u0.astype(np.float32)
    with Jacobi3D(dims, block, dtype=dtype, bc=BC_MIXED) as J:
        J.write(u0)
        for n in (0, 1, 9, 40):
            J.iterate(n)
            u = J.read(np.float32 if dtype == "f32" else np.float64)
            want = oracle.residual(u, BC_MIXED)
            got = J.residual()
            assert abs(got - want) <= 1e-12 * want


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_residual_slow_paths(dtype):
    """Residual parity where the frames do not hold every value: negative
    values, zeros, subnormals and exponent spreads wider than the binary64
    frame (31 binades: cells go to the exact per-cell list) and the binary32
    one (36 binades: the whole tile is redone exactly)."""
    dims, block = (34, 19, 13), (12, 7, 5)
    rng = np.random.default_rng(21)
    if dtype == "f64":
        u0 = rng.random(dims[::-1]) * 2.0 ** rng.integers(-80, 40, size=dims[::-1])
        u0.reshape(-1)[5::23] = 2.0 ** -1070
        bc = (3.0, -2.0, 1e-200, 0.0, -5e10, 7.0)
    else:
        u0 = (rng.random(dims[::-1]) * 2.0 ** rng.integers(-60, 30, size=dims[::-1])).astype(np.float32)
        u0.reshape(-1)[5::23] = np.float32(2.0 ** -140)
        bc = (3.0, -2.0, 1e-30, 0.0, -5e10, 7.0)
    u0 *= rng.choice([-1.0, 1.0], size=u0.shape).astype(u0.dtype)
    u0.reshape(-1)[::17] = 0.0
    with Jacobi3D(dims, block, dtype=dtype, bc=bc) as J:
        J.write(u0)
        for n in (0, 2):
            J.iterate(n)
            u = J.read(np.float32 if dtype == "f32" else np.float64)
            want = oracle.residual(u, bc)
            got = J.residual()
            assert abs(got - want) <= 1e-12 * want


def test_residual_of_fixed_point_is_zero():
    with Jacobi3D((12, 10, 8), (4, 5, 4), bc=(0.5,) * 6) as J:
        J.write(np.full((8, 10, 12), 0.5))
        J.iterate(3)
        assert J.residual() == 0.0
        assert np.all(J.read() == 0.5)


def test_zero_iterations_and_reread():
    dims = (10, 9, 8)
    u0 = grid(17, dims)
    with Jacobi3D(dims, (5, 3, 4), bc=BC_MIXED) as J:
        J.write(u0)
        J.iterate(0)
        assert np.array_equal(J.read(), u0)


@pytest.mark.parametrize("bad_value", [np.inf, -np.inf, np.nan, 2e300])
def test_write_rejects_bad_values_and_leaves_the_grid(bad_value):
    """Host and device writes check every value on the device before
    anything is overwritten: the error names the first bad index."""
    import torch

    with Jacobi3D((6, 5, 4), (3, 3, 2)) as J:
        good = synth.grid_uniform01(3, 6, 5, 4)
        J.write(good)
        bad = good.copy()
        bad[2, 3, 4] = bad_value  # flat index 2*30 + 3*6 + 4 = 82
        bad[3, 4, 5] = np.nan
        with pytest.raises(_lib.JacError) as e:
            J.write(bad)
        assert e.value.code == _lib.JAC_EINVAL and "82" in str(e.value)
        assert np.array_equal(J.read(), good)
        with pytest.raises(_lib.JacError) as e:
            J.write_device(torch.from_numpy(bad.reshape(-1)).cuda())
        assert e.value.code == _lib.JAC_EINVAL
        assert np.array_equal(J.read(), good)
    with Jacobi3D((6, 5, 4), (3, 3, 2), dtype="f32") as J:
        big = np.zeros((4, 5, 6))
        big[0, 0, 1] = 3.1e38  # finite in binary64, beyond the binary32 grid's range
        with pytest.raises(_lib.JacError):
            J.write(big)


def test_persistent_wait_timeout_reports_status_and_context_recovers():
    dims, block = (32, 16, 16), (8, 8, 8)
    u0 = grid(19, dims)
    with Jacobi3D(dims, block, bc=BC_MIXED, mode="persistent") as J:
        J.write(u0)
        _lib.jac_set_wait_limit_ns(J.h, 50_000_000)  # 50 ms
        _lib.jac_debug_withhold_progress(J.h, 5, 2)  # block 5 never reports iteration 2
        J.iterate(6)
        with pytest.raises(_lib.JacError) as e:
            J.sync()
        assert e.value.code == _lib.JAC_ETIMEOUT
        # the context stays usable
        _lib.jac_debug_withhold_progress(J.h, -1, 0)
        J.write(u0)
        J.iterate(4)
        got = J.read()
    assert np.array_equal(got, oracle.jacobi(u0, BC_MIXED, 4, oracle.RULE_EXACT))


def test_torch_stream_and_allocator():
    torch = pytest.importorskip("torch")
    from paper_2202_11819_gb300 import use_torch_allocator

    use_torch_allocator(True)
    try:
        dims = (24, 20, 16)
        u0 = grid(23, dims)
        s = torch.cuda.Stream()
        before = torch.cuda.memory_allocated()
        with torch.cuda.stream(s):
            with Jacobi3D(dims, (8, 10, 8), bc=BC_MIXED) as J:
                assert torch.cuda.memory_allocated() > before
                dev = torch.from_numpy(u0.reshape(-1)).to("cuda")
                J.write_device(dev)
                J.iterate(5)
                out = torch.empty_like(dev)
                J.read_device(out)
                rho = torch.zeros(1, dtype=torch.float64, device="cuda")
                J.residual_device(rho)
                s.synchronize()
        want = oracle.jacobi(u0, BC_MIXED, 5, oracle.RULE_EXACT)
        assert np.array_equal(out.cpu().numpy().reshape(want.shape), want)
        assert abs(rho.item() - oracle.residual(want, BC_MIXED)) <= 1e-12 * rho.item()
    finally:
        use_torch_allocator(False)


@pytest.mark.slow
@pytest.mark.parametrize("arith", ["exact", "seq"])
def test_full_size_512cubed_64cubed_blocks(arith):
    """The benchmark's launch configuration (512^3, 8x8x8 blocks of 64^3,
    persistent launch) against the oracle over the whole grid, a few
    iterations (the oracle's time is what bounds the count)."""
    dims, block = (512, 512, 512), (64, 64, 64)
    u0 = synth.grid_uniform01(0, *dims)
    n = 3
    want = oracle.jacobi(u0, synth.DIRICHLET_X0, n, ORACLE_RULE[arith])
    with Jacobi3D(dims, block, bc=synth.DIRICHLET_X0, mode="persistent", arith=arith) as J:
        J.write(u0)
        J.iterate(n)
        got = J.read()
        rho = J.residual()
    assert np.array_equal(got, want)
    assert abs(rho - oracle.residual(want, synth.DIRICHLET_X0)) <= 1e-12 * rho


@pytest.mark.slow
def test_full_size_forms_agree_and_invariants_hold():
    """All issue forms give identical grids at full size; after many
    iterations the maximum principle and residual decay still hold."""
    dims, block = (512, 512, 512), (64, 64, 64)
    u0 = synth.grid_uniform01(0, *dims)
    outs = {}
    for mode in ["fused", "persistent", "graph_fused"]:
        with Jacobi3D(dims, block, bc=synth.DIRICHLET_X0, mode=mode) as J:
            J.write(u0)
            r0 = J.residual()
            J.iterate(20)
            outs[mode] = J.read()
            r1 = J.residual()
            assert r1 < r0
    for m in outs:
        assert np.array_equal(outs[m], outs["persistent"])
    u = outs["persistent"]
    assert u.min() >= 0.0 and u.max() <= 1.0


def test_f32_error_against_f64_within_proven_bound():
    """Binary32 storage and arithmetic against the binary64 correctly rounded
    mean on the same grid: max|u32 - u64| <= k (27/7 + 1) 2^-24 + 2^-25."""
    dims, block = (96, 80, 72), (32, 40, 24)
    u0 = grid(29, dims)
    k = 300
    with Jacobi3D(dims, block, dtype="f32", bc=synth.DIRICHLET_X0, mode="persistent") as J:
        J.write(u0.astype(np.float32))
        J.iterate(k)
        u32 = J.read()
        r32 = J.residual()
    with Jacobi3D(dims, block, dtype="f64", bc=synth.DIRICHLET_X0, mode="persistent") as K:
        K.write(u0)
        K.iterate(k)
        u64 = K.read()
        r64 = K.residual()
    bound = k * (27.0 / 7.0 + 1.0) * 2.0 ** -24 + 2.0 ** -25
    err = np.max(np.abs(u32 - u64))
    assert 0 < err <= bound
    assert abs(r32 - r64) <= 0.05 * r64


@pytest.mark.parametrize("mode", ["unfused", "graph"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_unfused_forms_cover_tall_blocks(mode, dtype):
    """Per-block launches over blocks taller than one engine tile (64 rows,
    and binary32 work units of two engine tiles) update every row."""
    dims, block = (64, 64, 12), (64, 64, 6)
    u0 = grid(31, dims)
    if dtype == "f32":
        u0 = u0.astype(np.float32)
        want = oracle.jacobi_f32(u0, BC_MIXED, 4)
    else:
        want = oracle.jacobi(u0, BC_MIXED, 4, oracle.RULE_EXACT)
    got, _ = run(u0, dims, block, 4, mode, bc=BC_MIXED, dtype=dtype)
    assert np.array_equal(got, want)


_SEQ_1000 = {}


def _seq_oracle_1000(dims):
    # the left-to-right oracle at the benchmark's iteration count, computed
    # once per grid for the forms that compare with it
    if dims not in _SEQ_1000:
        u0 = synth.grid_uniform01(0, *dims)
        _SEQ_1000[dims] = (u0, oracle.jacobi(u0, synth.DIRICHLET_X0, 1000, oracle.RULE_SEQ))
    return _SEQ_1000[dims]


@pytest.mark.parametrize("mode", ["fused", "persistent"])
def test_exact_rule_within_1e12_relative_of_sequential_oracle_at_1000_iterations(mode):
    """The benchmark's rule (correctly rounded mean), blocks (64^3), boundary
    values and seed, at its 1000 iterations per step, against the
    left-to-right oracle element by element: |u - u_seq| <= 1e-12 |u_seq|.
    For non-negative data each rule stays within 7 units of roundoff of the
    exact mean relative to the cell value, so n iterations differ by at most
    n * 8 * 2^-53 = 8.9e-13 relative at n = 1000."""
    dims, block = (192, 128, 128), (64, 64, 64)
    u0, want = _seq_oracle_1000(dims)
    got, _ = run(u0, dims, block, 1000, mode, "exact")
    assert not np.array_equal(got, want)  # the two rules do round differently
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want))


def _tiles(info, dims, block):
    tw = info["tile_w"]
    th = 512 // tw  # binary64 work units: TW x 512/TW columns
    zd = info["zdepth"] if info["zdepth"] > 0 else block[2]
    nb = [-(-dims[a] // block[a]) for a in range(3)]
    per = -(-block[0] // tw) * -(-block[1] // th) * -(-block[2] // zd)
    return nb[0] * nb[1] * nb[2] * per


def test_last_wave_split_in_z_gives_the_oracle_result():
    """The runtime splits the units of a last wave it would leave at most half
    full in z. Grids where the split fires and where it does not must both
    match the oracle bit for bit, in the fused and persistent forms."""
    block = (64, 64, 64)
    seen = {True: 0, False: 0}
    for dims in [(128, 64, 64), (320, 320, 64), (64, 64, 128), (448, 448, 64)]:
        u0 = grid(37, dims)
        want = oracle.jacobi(u0, BC_MIXED, 3, oracle.RULE_EXACT)
        for mode in ("fused", "persistent"):
            with Jacobi3D(dims, block, bc=BC_MIXED, mode=mode) as J:
                J.write(u0)
                J.iterate(3)
                got = J.read()
                info = J.info()
            split = info["n_units"] > _tiles(info, dims, block)
            assert info["n_units"] >= _tiles(info, dims, block)
            seen[split] += 1
            assert np.array_equal(got, want), (dims, mode, split)
    assert seen[True] > 0 and seen[False] > 0, seen


@pytest.mark.parametrize("mode", ["fused", "persistent", "graph_fused"])
def test_per_tile_frames_on_blocks_of_very_different_magnitude(mode):
    """Each tile of the exact mean takes its fixed-point frame from the
    largest exponent among the values of its block and neighbours (written by
    the previous iteration), not from the grid's largest value. Blocks whose
    values lie many binades apart, a boundary value far above them, and a
    mode change and a rewrite in the middle, against the oracle bit for bit."""
    dims, block = (128, 128, 64), (32, 64, 32)
    u0 = grid(41, dims)
    # scale the eight blocks by 2^0, 2^-6, ..., 2^-42
    for bk in range(2):
        for bj in range(2):
            for bi in range(4):
                s = 2.0 ** (-6 * (bi + 4 * (bj + 2 * bk)))
                u0[bk * 32:(bk + 1) * 32, bj * 64:(bj + 1) * 64, bi * 32:(bi + 1) * 32] *= s
    bc = (2.0 ** 10, 0.0, 2.0 ** -30, 0.0, 1e-3, 0.5)
    want = oracle.jacobi(u0, bc, 12, oracle.RULE_EXACT)
    with Jacobi3D(dims, block, bc=bc, mode=mode) as J:
        J.write(u0)
        J.iterate(5)
        J.set_mode("unfused")  # a form that does not keep the per-unit bounds
        J.iterate(1)
        J.set_mode(mode)
        J.iterate(6)
        got = J.read()
        J.write(u0)  # the bounds of the old state must not survive a write
        J.iterate(12)
        got2 = J.read()
    assert np.array_equal(got, want)
    assert np.array_equal(got2, want)


@pytest.mark.parametrize("mode", ["fused", "persistent"])
@pytest.mark.parametrize("tile_w,zdepth", [(64, 0), (32, 0), (16, 0), (32, 12), (64, 7)])
def test_unit_frames_with_magnitudes_varying_inside_blocks(mode, tile_w, zdepth):
    """Each tile's frame comes from the exponent bounds of the units whose
    values it reads (its own, the adjacent units of its block, the face
    units of the neighbouring blocks) and the Dirichlet faces it touches.
    Magnitudes that change by 2^10 from one tile row, tile column or z slab
    to the next, inside blocks and across them, with several tile widths and
    z depths (units split in z), against the oracle bit for bit: a source
    left out of a list would put a value above its tile's frame."""
    dims, block = (96, 80, 60), (48, 40, 30)
    u0 = grid(43, dims)
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    expo = -10 * ((x // 16) % 3 + (y // 4) % 3 + (z // 6) % 3)
    u0 = u0 * 2.0 ** expo
    bc = (2.0 ** 8, 0.0, 2.0 ** -40, 0.25, 0.0, 1e-20)
    want = oracle.jacobi(u0, bc, 9, oracle.RULE_EXACT)
    with Jacobi3D(dims, block, bc=bc, mode=mode) as J:
        _lib.jac_set_tile(J.h, tile_w, zdepth)
        J.write(u0)
        J.iterate(9)
        got = J.read()
    assert np.array_equal(got, want)
