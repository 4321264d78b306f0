"""Serving runtime (include/irk_serve.h): continuous batching on one GPU.

Each request's result must be the same alone and in the mix (tolerance
1e-12 relative; the solver's reductions are per-handle and deterministic,
so in practice the results are bit-equal), admission must respect the HBM
budget, and a served request must still match the FP64 oracle.
"""
import threading
import time

import numpy as np
import pytest

import workloads
from oracle import irk as orc
from oracle.operators import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX_TOL = 1e-12


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01776_gb300 import build
    build.build()
    from paper_2101_01776_gb300 import binding
    return binding


def request_mix(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        n = int(rng.choice([32, 64, 128]))
        s = int(rng.choice([2, 3, 4]))
        nu = float(np.exp(rng.uniform(np.log(1e-3), np.log(1e-1))))
        out.append(dict(n=n, s=s, nu=nu, u0=workloads.random_fourier_2d(n, seed=100 + r)))
    return out


def alone(B, req, dt, nsteps):
    with B.IrkSolver(req["u0"], op="burgers2d", n=req["n"], stages=req["s"], nu=req["nu"]) as sol:
        sol.step(0.0, dt, nsteps)
        return sol.state()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_mix_equals_alone_and_stats(B):
    dt, nsteps = 1e-3, 4
    reqs = request_mix(10, seed=3)
    srv = B.irk_server_create(4, 2 << 30)
    try:
        ids = []
        for q in reqs:
            cfg = B.irk_config_default(op="burgers2d", n=q["n"], stages=q["s"], nu=q["nu"])
            ids.append(B.irk_server_submit(srv, cfg, q["u0"], 0.0, dt, nsteps))
        served = [B.irk_server_wait(srv, i, q["u0"].shape, nsteps) for i, q in zip(ids, reqs)]
        st = B.irk_server_stats_get(srv)
    finally:
        B.irk_server_destroy(srv)
    assert st["completed"] == 10 and st["failed"] == 0 and st["steps"] == 10 * nsteps
    assert 1 <= st["peak_active"] <= 4
    assert st["p50_step_ms"] <= st["p99_step_ms"] <= st["max_step_ms"]
    assert st["peak_bytes"] <= st["budget_bytes"]
    for q, (u, stats, ms) in zip(reqs, served):
        assert stats.steps == nsteps and len(ms) == nsteps and np.all(ms > 0)
        assert rel(u, alone(B, q, dt, nsteps)) <= MIX_TOL


def test_admission_is_bounded_by_the_hbm_budget(B):
    dt, nsteps = 1e-3, 2
    cfg = B.irk_config_default(op="burgers2d", n=128, stages=4, nu=1e-2)
    need = B.irk_config_device_bytes(cfg)
    srv = B.irk_server_create(4, int(need * 1.5))  # room for one request at a time
    try:
        u0 = workloads.random_fourier_2d(128, seed=1)
        ids = [B.irk_server_submit(srv, cfg, u0, 0.0, dt, nsteps) for _ in range(3)]
        outs = [B.irk_server_wait(srv, i, u0.shape, nsteps)[0] for i in ids]
        st = B.irk_server_stats_get(srv)
        big = B.irk_config_default(op="burgers2d", n=512, stages=4, nu=1e-2)
        with pytest.raises(B.IrkError) as ei:
            B.irk_server_submit(srv, big, workloads.random_fourier_2d(512, seed=1), 0.0, dt, 1)
        assert ei.value.status == B.IRK_ERR_NOMEM
    finally:
        B.irk_server_destroy(srv)
    assert st["peak_active"] == 1
    assert st["peak_bytes"] <= st["budget_bytes"]
    for u in outs[1:]:
        np.testing.assert_array_equal(u, outs[0])


def test_requests_arriving_while_others_run(B):
    """A producer thread submits with random gaps (Poisson arrivals) while
    earlier requests are on the GPU; each result still equals its solo run,
    and a served 2D Burgers request matches the FP64 oracle."""
    dt, nsteps = 1e-3, 3
    reqs = request_mix(8, seed=11)
    srv = B.irk_server_create(3, 2 << 30)
    ids = [None] * len(reqs)
    rng = np.random.default_rng(0)

    def producer():
        for k, q in enumerate(reqs):
            cfg = B.irk_config_default(op="burgers2d", n=q["n"], stages=q["s"], nu=q["nu"])
            ids[k] = B.irk_server_submit(srv, cfg, q["u0"], 0.0, dt, nsteps)
            time.sleep(float(rng.exponential(0.01)))
    try:
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        served = [B.irk_server_wait(srv, i, q["u0"].shape, nsteps)[0] for i, q in zip(ids, reqs)]
    finally:
        B.irk_server_destroy(srv)
    for q, u in zip(reqs, served):
        assert rel(u, alone(B, q, dt, nsteps)) <= MIX_TOL
    k = min(range(len(reqs)), key=lambda i: reqs[i]["n"] * reqs[i]["s"])
    q = reqs[k]
    p = Problem("burgers2d", q["n"], q["nu"])
    ref, _ = orc.integrate(p, q["s"], q["u0"], 0.0, dt, nsteps)
    assert rel(served[k], ref) <= 1e-8


def test_served_families_and_dae_solver_equal_alone(B):
    """Requests of every tableau family and the VSF forward solve through the
    server: a stage-by-stage SDIRK handle carves its single-stage solver out of
    the arena the server hands it, and each result equals its solo run."""
    import math
    dt, nsteps = 1e-3, 2
    specs = [dict(op="burgers2d", n=64, stages=3, nu=1e-2, family="sdirk"),
             dict(op="burgers2d", n=64, stages=5, nu=1e-2, family="sdirk", dirk_sequential=0),
             dict(op="burgers2d", n=32, stages=3, nu=1e-2, family="radau"),
             dict(op="burgers2d", n=32, stages=3, nu=1e-2, family="lobatto"),
             dict(op="vsf", n=32, stages=2, nu=1e-3, length=2 * math.pi, dae_solver=1),
             dict(op="vsf", n=32, stages=2, nu=1e-3, length=2 * math.pi, family="sdirk")]
    u0s = []
    for k, sp in enumerate(specs):
        if sp["op"] == "vsf":
            u = np.zeros((2, sp["n"], sp["n"]))
            u[0] = workloads.double_shear_layer_vorticity(sp["n"], seed=k)
        else:
            u = workloads.random_fourier_2d(sp["n"], seed=200 + k)
        u0s.append(u)
    srv = B.irk_server_create(3, 2 << 30)
    try:
        ids = [B.irk_server_submit(srv, B.irk_config_default(**sp), u, 0.0, dt, nsteps)
               for sp, u in zip(specs, u0s)]
        served = [B.irk_server_wait(srv, i, u.shape, nsteps) for i, u in zip(ids, u0s)]
        st = B.irk_server_stats_get(srv)
    finally:
        B.irk_server_destroy(srv)
    assert st["completed"] == len(specs) and st["failed"] == 0
    for sp, u0, (u, stats, _) in zip(specs, u0s, served):
        with B.IrkSolver(u0, **sp) as sol:
            sol.step(0.0, dt, nsteps)
            ref = sol.state()
        assert stats.steps == nsteps
        assert rel(u, ref) <= MIX_TOL, sp


def served_batched(B, reqs, dt, nsteps, capacity, gaps=None):
    srv = B.irk_server_create_batched(capacity, 2 << 30)
    try:
        ids = []
        for k, q in enumerate(reqs):
            cfg = B.irk_config_default(op="burgers2d", n=q["n"], stages=q["s"], nu=q["nu"])
            ids.append(B.irk_server_submit(srv, cfg, q["u0"], 0.0, dt, nsteps))
            if gaps is not None:
                time.sleep(float(gaps[k]))
        out = [B.irk_server_wait(srv, i, q["u0"].shape, nsteps) for i, q in zip(ids, reqs)]
        st = B.irk_server_stats_get(srv)
    finally:
        B.irk_server_destroy(srv)
    return out, st


def test_batched_server_mix_equals_alone_and_oracle(B):
    """The batched server (one graph launch per step for all residents):
    requests arriving while others run give bit for bit the result they give
    alone in the batched server, and a served request matches the oracle."""
    dt, nsteps = 1e-3, 4
    reqs = request_mix(9, seed=5)
    gaps = np.random.default_rng(1).exponential(0.005, size=len(reqs))
    served, st = served_batched(B, reqs, dt, nsteps, capacity=4, gaps=gaps)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["steps"] == len(reqs) * nsteps and 1 <= st["peak_active"] <= 4
    assert st["p50_step_ms"] <= st["p99_step_ms"] <= st["max_step_ms"]
    for q, (u, stats, ms) in zip(reqs, served):
        assert stats.steps == nsteps and len(ms) == nsteps
        (u1, _, _), = served_batched(B, [q], dt, nsteps, capacity=1)[0]
        assert np.array_equal(u, u1)
    k = min(range(len(reqs)), key=lambda i: reqs[i]["n"] * reqs[i]["s"])
    q = reqs[k]
    ref, _ = orc.integrate(Problem("burgers2d", q["n"], q["nu"]), q["s"], q["u0"], 0.0, dt, nsteps)
    assert rel(served[k][0], ref) <= 1e-8


def test_batched_server_rejects_what_the_batch_does_not_serve(B):
    srv = B.irk_server_create_batched(2, 1 << 30)
    try:
        cfg = B.irk_config_default(op="burgers1d", n=64, stages=2, nu=1e-2)
        with pytest.raises(B.IrkError) as ei:
            B.irk_server_submit(srv, cfg, np.zeros((1, 64)), 0.0, 1e-3, 2)
        assert ei.value.status == B.IRK_ERR_INVALID
    finally:
        B.irk_server_destroy(srv)


def test_hybrid_server_batches_small_grids_and_streams_large_ones(B):
    """The batched server with stream workers for n >= 128: the 32^2/64^2
    requests run in the batch (bit for bit their result alone in a batch),
    the 128^2 ones on their own streams (their single-instance result)."""
    dt, nsteps = 1e-3, 3
    reqs = request_mix(8, seed=9)
    assert any(q["n"] >= 128 for q in reqs) and any(q["n"] < 128 for q in reqs)
    srv = B.irk_server_create_batched(4, 2 << 30, stream_slots=2, stream_min_n=128)
    try:
        ids = [B.irk_server_submit(srv, B.irk_config_default(op="burgers2d", n=q["n"], stages=q["s"],
                                                             nu=q["nu"]), q["u0"], 0.0, dt, nsteps)
               for q in reqs]
        served = [B.irk_server_wait(srv, i, q["u0"].shape, nsteps)[0] for i, q in zip(ids, reqs)]
        st = B.irk_server_stats_get(srv)
    finally:
        B.irk_server_destroy(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for q, u in zip(reqs, served):
        if q["n"] >= 128:
            assert rel(u, alone(B, q, dt, nsteps)) <= MIX_TOL
        else:
            (u1, _, _), = served_batched(B, [q], dt, nsteps, capacity=1)[0]
            assert np.array_equal(u, u1)
