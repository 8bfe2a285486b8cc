"""Batched contexts (several grids in one pool and one launch), tile shapes,
z depths and the autotuner, against the CPU oracle run on each grid alone.

Tolerances as in test_parity_gpu: binary64 bit-exact against the matching
oracle rule, binary32 bit-exact, residuals 1e-12 relative.
"""

import numpy as np
import pytest

import oracle
import synth
from paper_2202_11819_gb300 import Jacobi3DBatch, _lib

pytestmark = pytest.mark.gpu

RULE = {"seq": oracle.RULE_SEQ, "exact": oracle.RULE_EXACT}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.load()


def instance_set(n, seed, lo=5, hi=41):
    rng = np.random.default_rng(seed)
    dims = [tuple(int(v) for v in rng.integers(lo, hi, size=3)) for _ in range(n)]
    bcs = [tuple(float(v) for v in rng.random(6)) for _ in range(n)]
    grids = [synth.grid_uniform01(100 + i, *d).copy() for i, d in enumerate(dims)]
    return dims, bcs, grids


@pytest.mark.parametrize("arith", ["exact", "seq"])
@pytest.mark.parametrize("mode", ["persistent", "fused", "unfused", "graph_fused"])
def test_batch_matches_each_grid_alone(mode, arith):
    dims, bcs, grids = instance_set(6, 1)
    iters = 7
    with Jacobi3DBatch(dims, (16, 12, 10), bcs=bcs, mode=mode, arith=arith) as B:
        for i, g in enumerate(grids):
            B.write(i, g)
        B.iterate(iters)
        outs = [B.read(i) for i in range(len(dims))]
        rhos = B.residuals()
    for i, g in enumerate(grids):
        want = oracle.jacobi(g, bcs[i], iters, RULE[arith])
        assert np.array_equal(outs[i], want), f"grid {i}"
        r = oracle.residual(want, bcs[i])
        assert abs(rhos[i] - r) <= 1e-12 * r


@pytest.mark.parametrize("tile_w", [16, 32, 64])
@pytest.mark.parametrize("zdepth", [0, 16, 7])
@pytest.mark.parametrize("mode", ["persistent", "fused"])
def test_tile_shapes_and_z_depths_do_not_change_results(tile_w, zdepth, mode):
    dims, bcs, grids = instance_set(3, 2, lo=9, hi=80)
    iters = 5
    with Jacobi3DBatch(dims, (64, 40, 33), bcs=bcs, mode=mode) as B:
        B.set_tile(tile_w, zdepth)
        info = B.info()
        assert info["tile_w"] == tile_w and info["zdepth"] == zdepth
        for i, g in enumerate(grids):
            B.write(i, g)
        B.iterate(iters)
        outs = [B.read(i) for i in range(len(dims))]
        rhos = B.residuals()
    for i, g in enumerate(grids):
        want = oracle.jacobi(g, bcs[i], iters, oracle.RULE_EXACT)
        assert np.array_equal(outs[i], want), f"grid {i}"
        assert abs(rhos[i] - oracle.residual(want, bcs[i])) <= 1e-12 * rhos[i]


def test_f32_batch():
    dims, bcs, grids = instance_set(4, 3)
    iters = 6
    with Jacobi3DBatch(dims, (16, 16, 16), dtype="f32", bcs=bcs, mode="persistent") as B:
        for i, g in enumerate(grids):
            B.write(i, g)
        B.iterate(iters)
        outs = [B.read(i) for i in range(len(dims))]
    for i, g in enumerate(grids):
        want = oracle.jacobi_f32(g.astype(np.float32), bcs[i], iters).astype(np.float64)
        assert np.array_equal(outs[i], want), f"grid {i}"


def test_autotune_restores_state_and_keeps_results():
    dims, bcs, grids = instance_set(5, 4, lo=20, hi=70)
    with Jacobi3DBatch(dims, (32, 32, 32), bcs=bcs, mode="persistent") as B:
        for i, g in enumerate(grids):
            B.write(i, g)
        B.iterate(3)
        before = [B.read(i) for i in range(len(dims))]
        it_before = B.info()["iterations"]
        res = B.autotune(2)
        assert res["tile_w"] in (16, 32, 64)
        assert len(res["trials"]) >= 3
        assert B.info()["iterations"] == it_before
        after = [B.read(i) for i in range(len(dims))]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        B.iterate(4)
        outs = [B.read(i) for i in range(len(dims))]
    for i, g in enumerate(grids):
        assert np.array_equal(outs[i], oracle.jacobi(g, bcs[i], 7, oracle.RULE_EXACT))


def test_rewriting_one_grid_leaves_the_others():
    dims, bcs, grids = instance_set(4, 5)
    with Jacobi3DBatch(dims, (16, 16, 16), bcs=bcs) as B:
        for i, g in enumerate(grids):
            B.write(i, g)
        B.iterate(4)
        fresh = synth.grid_uniform01(999, *dims[2]).copy()
        B.write(2, fresh)
        B.iterate(3)
        outs = [B.read(i) for i in range(len(dims))]
    for i, g in enumerate(grids):
        if i == 2:
            want = oracle.jacobi(fresh, bcs[i], 3, oracle.RULE_EXACT)
        else:
            want = oracle.jacobi(g, bcs[i], 7, oracle.RULE_EXACT)
        assert np.array_equal(outs[i], want), f"grid {i}"


def test_batch_of_configured_shapes_small():
    """Shapes drawn as the batched workload draws them (each axis from
    32, 48, ..., 192), a few grids, blocks of at most 64^3, parity on a
    few sampled grids."""
    dims = synth.batch_instance_dims(6, seed=0)
    grids = [synth.grid_uniform01(i, *d) for i, d in enumerate(dims)]
    bc = synth.DIRICHLET_X0
    with Jacobi3DBatch(dims, (64, 64, 64), bcs=[bc] * len(dims), mode="persistent") as B:
        for i, g in enumerate(grids):
            B.write(i, g)
        B.iterate(3)
        for i in (0, 3):
            assert np.array_equal(B.read(i), oracle.jacobi(grids[i], bc, 3, oracle.RULE_EXACT))


@pytest.mark.parametrize("tile_w", [16, 32, 64])
@pytest.mark.parametrize("zdepth", [0, 16, 7])
@pytest.mark.parametrize("mode", ["persistent", "fused"])
def test_f32_tile_shapes_and_z_depths_bit_exact(tile_w, zdepth, mode):
    """The binary32 ring engine over ragged blocks (tiles overhanging block
    edges), z ranges shorter than a ring turn (zdepth 7, 16) and whole 64-plane
    blocks (whole ring turns without range checks), against the binary32
    oracle."""
    dims = [(70, 45, 100), (17, 64, 64), (64, 9, 131)]
    rng = np.random.default_rng(6)
    bcs = [tuple(float(v) for v in rng.random(6)) for _ in dims]
    grids = [synth.grid_uniform01(300 + i, *d).astype(np.float32) for i, d in enumerate(dims)]
    iters = 5
    with Jacobi3DBatch(dims, (64, 40, 64), dtype="f32", bcs=bcs, mode=mode) as B:
        B.set_tile(tile_w, zdepth)
        for i, g in enumerate(grids):
            _lib.jac_write_instance(B.h, i, g.astype(np.float64))
        B.iterate(iters)
        outs = [B.read(i) for i in range(len(dims))]
    for i, g in enumerate(grids):
        want = oracle.jacobi_f32(g, bcs[i], iters).astype(np.float64)
        assert np.array_equal(outs[i], want), f"grid {i}"


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mode", ["persistent", "fused"])
def test_per_class_tile_widths_bit_exact(dtype, mode):
    """Blocks of different x extents (35, 40, 50) run with different tile
    widths in one launch; results stay those of the oracle."""
    dims = [(70, 45, 50), (40, 64, 30), (100, 33, 41)]
    rng = np.random.default_rng(21)
    bcs = [tuple(float(v) for v in rng.random(6)) for _ in dims]
    grids = [synth.grid_uniform01(400 + i, *d) for i, d in enumerate(dims)]
    if dtype == "f32":
        grids = [g.astype(np.float32).astype(np.float64) for g in grids]
    iters = 5
    with Jacobi3DBatch(dims, (64, 40, 64), dtype=dtype, bcs=bcs, mode=mode) as B:
        B.set_tile(32, 0)
        B.set_tile_class(35, 16)
        B.set_tile_class(50, 64)
        for i, g in enumerate(grids):
            B.write(i, g)
        B.iterate(iters)
        outs = [B.read(i) for i in range(len(dims))]
        rhos = B.residuals()
    for i, g in enumerate(grids):
        if dtype == "f32":
            want = oracle.jacobi_f32(g.astype(np.float32), bcs[i], iters).astype(np.float64)
            assert np.array_equal(outs[i], want), f"grid {i}"
            # a binary32 grid's boundary values are stored in binary32
            r = oracle.residual(want, tuple(float(np.float32(v)) for v in bcs[i]))
        else:
            want = oracle.jacobi(g, bcs[i], iters, oracle.RULE_EXACT)
            assert np.array_equal(outs[i], want), f"grid {i}"
            r = oracle.residual(want, bcs[i])
        assert abs(rhos[i] - r) <= 1e-12 * r


def test_autotune_refines_block_width_classes():
    dims = synth.batch_instance_dims(12, seed=3)
    grids = [synth.grid_uniform01(i, *d) for i, d in enumerate(dims)]
    bc = synth.DIRICHLET_X0
    with Jacobi3DBatch(dims, (64, 64, 64), bcs=[bc] * len(dims), mode="persistent") as B:
        for i, g in enumerate(grids):
            B.write(i, g)
        res = B.autotune(2)
        widths = {d[0] if d[0] <= 64 else -(-d[0] // -(-d[0] // 64)) for d in dims}
        if len(widths) > 1:
            assert res.get("classes"), res
            assert all(tw in (16, 32, 64) for _, tw in res["classes"])
        B.iterate(3)
        for i in (0, 5, 11):
            assert np.array_equal(B.read(i), oracle.jacobi(grids[i], bc, 3, oracle.RULE_EXACT))
