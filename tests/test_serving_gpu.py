"""Pools (grids joining and leaving between launches) and the solve server
(continuous batching): every result is the same as the oracle's for that
grid alone and the same whether the request ran alone or in the mix.

Tolerances: bit-exact (binary64 correctly rounded mean and binary32 both
match their oracle rules exactly, and a grid's arithmetic never involves
another grid's cells).
"""

import numpy as np
import pytest

import oracle
import synth
from paper_2202_11819_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.load()


def oracle_run(u0, bc, iters, dtype):
    if dtype == _lib.JAC_F32:
        return oracle.jacobi_f32(u0.astype(np.float32), bc, iters).astype(np.float64)
    return oracle.jacobi(u0, bc, iters, oracle.RULE_EXACT)


def test_pool_grids_join_and_leave_between_launches():
    rng = np.random.default_rng(3)
    h = _lib.jac_create_pool(_lib.JAC_F64, 64 << 20, 8, 16, 16, 16)
    try:
        grids, slots, iters = {}, {}, {}
        for step in range(5):
            # a new grid joins
            d = tuple(int(v) for v in rng.integers(6, 40, size=3))
            bc = tuple(float(v) for v in rng.random(6))
            u = synth.grid_uniform01(50 + step, *d).copy()
            s = _lib.jac_pool_add(h, d, bc)
            _lib.jac_write_instance(h, s, u)
            grids[s], iters[s] = (d, bc, u), 0
            # an old one leaves
            if step == 3:
                victim = sorted(grids)[0]
                _lib.jac_pool_remove(h, victim)
                del grids[victim], iters[victim]
            _lib.jac_iterate(h, 3)
            for k in iters:
                iters[k] += 3
        used, cap, n = _lib.jac_pool_usage(h)
        assert n == len(grids) and 0 < used <= cap
        rho = _lib.jac_residual_instances(h, max(grids) + 1)
        for s, (d, bc, u) in grids.items():
            got = _lib.jac_read_instance(h, s, np.empty(d[::-1]))
            want = oracle_run(u, bc, iters[s], _lib.JAC_F64)
            assert np.array_equal(got, want), f"slot {s}"
            assert abs(rho[s] - oracle.residual(want, bc)) <= 1e-12 * rho[s]
    finally:
        _lib.jac_destroy(h)


def test_pool_rejects_grids_beyond_capacity():
    h = _lib.jac_create_pool(_lib.JAC_F64, 4 << 20, 4, 32, 32, 32)
    try:
        with pytest.raises(_lib.JacError) as e:
            _lib.jac_pool_add(h, (200, 200, 200), (0,) * 6)
        assert e.value.code == _lib.JAC_EBUDGET
    finally:
        _lib.jac_destroy(h)


REQUESTS = [
    # dims, dtype, tol, max_iters
    ((4, 5, 6), _lib.JAC_F64, 1e-6, 600),     # converges well before the cap
    ((40, 33, 21), _lib.JAC_F64, 1e-6, 200),  # hits the cap
    ((17, 9, 30), _lib.JAC_F32, 1e-6, 150),
    ((6, 6, 6), _lib.JAC_F32, 1e-5, 600),
    ((64, 20, 12), _lib.JAC_F64, 1e-9, 100),
    ((25, 25, 25), _lib.JAC_F32, 1e-6, 250),
]


def run_server(reqs, budget, max_active, arrivals=None, chunk=25):
    s = _lib.jac_server_create(budget, max_active, 16, 16, 16, chunk)
    out = {}
    try:
        ids = {}
        pending = list(range(len(reqs)))
        steps = 0
        while pending or len(out) < len(reqs):
            # staggered arrivals: request i is submitted at step arrivals[i]
            for i in list(pending):
                if arrivals is None or arrivals[i] <= steps:
                    dims, dtype, tol, cap, u0, bc = reqs[i]
                    ids[_lib.jac_server_submit(s, dims, dtype, bc, u0, tol, cap)] = i
                    pending.remove(i)
            _lib.jac_server_step(s)
            steps += 1
            while True:
                r = _lib.jac_server_poll(s)
                if r is None:
                    break
                i = ids[r["id"]]
                assert r["status"] == 0
                res = _lib.jac_server_result(s, r["id"], np.empty(reqs[i][0][::-1]))
                out[i] = (res, r["iterations"], r["residual"])
            assert steps < 10000
    finally:
        _lib.jac_server_destroy(s)
    return out


def request_set():
    rs = []
    for i, (dims, dtype, tol, cap) in enumerate(REQUESTS):
        u0 = synth.grid_uniform01(200 + i, *dims).copy()
        bc = (1.0, 0.0, 0.25, 0.0, 0.5, 0.0)
        rs.append((dims, dtype, tol, cap, u0, bc))
    return rs


def test_server_results_same_alone_and_in_the_mix():
    reqs = request_set()
    mixed = run_server(reqs, 256 << 20, 4, arrivals=[0, 0, 1, 3, 4, 9])
    for i, rq in enumerate(reqs):
        alone = run_server([rq], 256 << 20, 1)[0]
        res, it, rho = mixed[i]
        assert np.array_equal(res, alone[0]), f"request {i}"
        assert it == alone[1] and rho == alone[2]
        # and the oracle for that many iterations agrees
        dims, dtype, tol, cap, u0, bc = rq
        assert np.array_equal(res, oracle_run(u0, bc, it, dtype))
        assert it % 25 == 0 and it <= cap
        assert rho < tol or it == cap


def test_server_admission_waits_for_budget():
    reqs = request_set()
    need = max(_lib.jac_storage_bytes(r[0], 16, 16, 16, r[1]) for r in reqs)
    # room for one grid at a time: everything still finishes, one after another
    out = run_server(reqs, need + 4096, 8)
    assert len(out) == len(reqs)
    for i, rq in enumerate(reqs):
        dims, dtype, tol, cap, u0, bc = rq
        res, it, rho = out[i]
        assert np.array_equal(res, oracle_run(u0, bc, it, dtype))


def test_server_rejects_oversized_request():
    s = _lib.jac_server_create(1 << 20, 4, 16, 16, 16, 10)
    try:
        with pytest.raises(_lib.JacError) as e:
            _lib.jac_server_submit(s, (128, 128, 128), _lib.JAC_F64, (0,) * 6, np.zeros(128 ** 3), 1e-6, 10)
        assert e.value.code == _lib.JAC_EBUDGET
    finally:
        _lib.jac_server_destroy(s)
