"""The batched path (include/irk_batch.h) against the oracle, and mix == alone.

Instances of different grid sizes, stage counts and viscosities share every
kernel launch of a step.  Each instance must still compute Algorithm 1's
fixed point of its own stage equations (Sec. 1.1 Eq. stages/update): per
step, starting from the GPU's u_n, u_{n+1} matches the oracle's step from
that u_n within 1e-9 relative L2, and the stages satisfy the oracle's stage
residual to the Newton tolerance.  Per-instance reductions are summed over
that instance's own chunks in a fixed order, so an instance's states are bit
for bit the same alone and in any mix, also across admissions and removals
that change the launch structure.
"""
import numpy as np
import pytest

import workloads
from oracle import irk as orc
from oracle import tableau as tab
from oracle.operators import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP_TOL = 1e-9


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01776_gb300 import build
    build.build()
    from paper_2101_01776_gb300 import binding
    return binding


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# (n, s, nu, dt, seed): uneven sizes, stage counts and viscosities
MIX = [(32, 2, 1e-2, 1e-3, 1), (64, 3, 3e-3, 1e-3, 2), (32, 4, 5e-2, 1e-3, 3), (64, 1, 1e-3, 2e-3, 4),
       (64, 2, 2e-2, 1e-3, 5)]


def oracle_step(n, s, nu, u, dt):
    p = Problem("burgers2d", n, nu)
    linear = "direct" if p.size * s <= 40000 else "gmres"
    return orc.step(p, s, u, 0.0, dt, linear=linear)


def test_batched_mix_matches_oracle_per_step(B):
    with B.IrkBatch(8) as bt:
        slots = []
        for (n, s, nu, dt, seed) in MIX:
            u0 = workloads.random_fourier_2d(n, seed=seed)
            slots.append(bt.add(u0, dt, op="burgers2d", n=n, stages=s, nu=nu))
        for step in range(3):
            before = {k: bt.state(k).copy() for k in slots}
            res = bt.step()
            for k, (n, s, nu, dt, seed) in zip(slots, MIX):
                status, st = res[k]
                assert status == 0 and st["steps"] == 1, (k, res[k])
                assert st["final_rel_res"] <= 1e-10, (k, st)
                got = bt.state(k)
                K = bt.stages(k)
                p = Problem("burgers2d", n, nu)
                A, b, c = tab.gauss(s)
                F = orc.stage_residual(p, before[k], K, 0.0, dt, A, c)
                F0 = orc.stage_residual(p, before[k], np.zeros_like(K), 0.0, dt, A, c)
                assert np.linalg.norm(F) <= 2e-10 * np.linalg.norm(F0), (k, step)
                assert rel(got, before[k] + dt * np.tensordot(b, K, axes=(0, 0))) <= 1e-14
                want, _, _ = oracle_step(n, s, nu, before[k], dt)
                assert rel(got, want) <= STEP_TOL, (k, step, rel(got, want), st)


def test_batched_instance_is_bit_equal_alone_and_in_any_mix(B):
    """The same instance alone, in a mix, and in a mix that changes (another
    instance removed and two admitted between steps): equal bit for bit."""
    n, s, nu, dt = 64, 3, 3e-3, 1e-3
    u0 = workloads.random_fourier_2d(n, seed=11)
    with B.IrkBatch(4) as alone:
        k = alone.add(u0, dt, op="burgers2d", n=n, stages=s, nu=nu)
        for _ in range(4):
            alone.step()
        ref = alone.state(k).copy()
    with B.IrkBatch(6) as mix:
        others = [mix.add(workloads.random_fourier_2d(32, seed=20), 1e-3, op="burgers2d", n=32,
                          stages=2, nu=1e-2)]
        k = mix.add(u0, dt, op="burgers2d", n=n, stages=s, nu=nu)
        others.append(mix.add(workloads.random_fourier_2d(128, seed=21), 1e-3, op="burgers2d",
                              n=128, stages=4, nu=1e-3))
        mix.step()
        mix.step()
        mix.remove(others[0])
        mix.add(workloads.random_fourier_2d(64, seed=22), 2e-3, op="burgers2d", n=64, stages=5,
                nu=5e-3)
        mix.add(workloads.random_fourier_2d(32, seed=23), 1e-3, op="burgers2d", n=32, stages=1,
                nu=4e-2)
        mix.step()
        mix.step()
        got = mix.state(k)
    assert np.array_equal(got, ref)


def test_batched_matches_single_instance_solver(B):
    """The batched path and the single-instance solver reach the same fixed
    point (both to Newton relative residual 1e-10)."""
    n, s, nu, dt = 64, 2, 5e-3, 2e-3
    u0 = workloads.random_fourier_2d(n, seed=12)
    with B.IrkBatch(2) as bt:
        k = bt.add(u0, dt, op="burgers2d", n=n, stages=s, nu=nu)
        for _ in range(3):
            bt.step()
        got = bt.state(k)
    with B.IrkSolver(u0, op="burgers2d", n=n, stages=s, nu=nu) as sol:
        sol.step(0.0, dt, 3)
        want = sol.state()
    assert rel(got, want) <= 1e-9


def test_batched_failure_is_per_instance(B):
    """newton_maxit = 1 makes one instance fail: it keeps its state, reports
    IRK_ERR_NEWTON_MAXIT, and the others step normally."""
    with B.IrkBatch(4) as bt:
        u_bad = workloads.random_fourier_2d(32, seed=30)
        u_ok = workloads.random_fourier_2d(32, seed=31)
        kb = bt.add(u_bad, 5e-3, op="burgers2d", n=32, stages=2, nu=1e-2, newton_maxit=1)
        ko = bt.add(u_ok, 1e-3, op="burgers2d", n=32, stages=2, nu=1e-2)
        res = bt.step()
        assert res[kb][0] == B.IRK_ERR_NEWTON_MAXIT
        assert res[ko][0] == 0
        np.testing.assert_array_equal(bt.state(kb), u_bad)
        want, _, _ = oracle_step(32, 2, 1e-2, u_ok, 1e-3)
        assert rel(bt.state(ko), want) <= STEP_TOL


def test_batched_rejects_what_it_does_not_serve(B):
    with B.IrkBatch(2) as bt:
        u = np.zeros((2, 64, 64))
        with pytest.raises(B.IrkError) as ei:
            bt.add(u, 1e-3, op="burgers2d", n=64, stages=2, nu=1e-2, mg_precision=1)
        assert ei.value.status == B.IRK_ERR_INVALID
        # dt nu so large that no level of the hierarchy is shift dominated
        with pytest.raises(B.IrkError) as ei:
            bt.add(u, 1.0, op="burgers2d", n=64, stages=2, nu=10.0)
        assert ei.value.status == B.IRK_ERR_INVALID
        assert bt.count() == 0
        assert bt.step() == {}


def test_batched_zero_state_and_device_arena(B):
    """A zero state is solved by zero stages (no Newton iteration); an instance
    in a caller-owned device arena steps like one the batch allocates."""
    n, s, nu, dt = 32, 3, 1e-2, 1e-3
    u0 = workloads.random_fourier_2d(n, seed=40)
    cfg = B.irk_config_default(op="burgers2d", n=n, stages=s, nu=nu)
    nbytes = B.IrkBatch.instance_bytes(cfg)
    arena = torch.empty(nbytes // 8 + 64, dtype=torch.float64, device="cuda")
    ptr = (arena.data_ptr() + 255) // 256 * 256
    with B.IrkBatch(4) as bt:
        kz = bt.add(np.zeros((2, n, n)), dt, op="burgers2d", n=n, stages=s, nu=nu)
        ka = bt.add(torch.from_numpy(u0).cuda(), dt, arena_ptr=ptr, arena_bytes=nbytes,
                    op="burgers2d", n=n, stages=s, nu=nu)
        kb = bt.add(u0, dt, op="burgers2d", n=n, stages=s, nu=nu)
        for _ in range(2):
            res = bt.step()
        assert res[kz][0] == 0 and res[kz][1]["newton_its"] == 0
        assert np.all(bt.state(kz) == 0)
        assert np.array_equal(bt.state(ka), bt.state(kb))
