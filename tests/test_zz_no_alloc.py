"""The allocation-free stage-residual entry point against the oracle.

irk_stage_residual_noalloc serves callers that cannot call cudaMalloc (a host
whose memory manager owns the device pool, a latency-critical loop that must
not synchronise the device through cudaMalloc/cudaFree, a fixed memory
budget).  Its scratch is a fixed file-scope device array shared by all calls,
so the calls here run back to back on it, and each is compared with the
oracle's stage residual (Eq. stages) and its 2-norm at the same 1e-12
tolerance as the other residual tests; the regular entry point, which uses a
handle's allocated buffers, must give the same F.  A larger grid runs before
a smaller one, so the second norm would read stale partials of the first if
it summed more slots than its own.  The file is named to be collected last.
"""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import irk as orc
from oracle import tableau as tab
from oracle.operators import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01776_gb300 import build
    build.build()
    from paper_2101_01776_gb300 import binding
    return binding


def _shape(op, n):
    return (2, n, n) if op in ("burgers2d", "vsf") else (1, n)


def _oracle(op, n, s, nu, length, dt, u, K):
    p = Problem(op, n, nu, length)
    A, _, c = tab.gauss(s)
    return orc.stage_residual(p, u, K, 0.0, dt, A, c)


def _regular(B, op, n, s, nu, length, dt, u, K):
    with B.IrkSolver(u, op=op, n=n, stages=s, nu=nu, length=length) as sol:
        sol.set_state(u)
        return B.irk_stage_residual(sol.h, 0.0, dt, K, np.empty_like(K))


def _noalloc(B, op, n, s, nu, length, dt, u, K):
    dev = torch.device("cuda", 0)
    A = B.irk_tableau(s)["A"]
    F = torch.full((s,) + _shape(op, n), float("nan"), dtype=torch.float64, device=dev)
    fnorm = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    ud = torch.from_numpy(u).to(dev)
    Kd = torch.from_numpy(K).to(dev)
    B.irk_stage_residual_noalloc(op, n, length, nu, s, A, dt, ud, Kd, F, fnorm,
                                 torch.cuda.current_stream(dev))
    torch.cuda.synchronize(dev)
    return F.cpu().numpy(), float(fnorm.item())


def _check(B, op, n, s, length, seed, against_regular=True):
    nu, dt = 0.011, 2.5e-3
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(_shape(op, n))
    K = rng.standard_normal((s,) + _shape(op, n)) * (1 + seed % 3)
    want = _oracle(op, n, s, nu, length, dt, u, K)
    got, fnorm = _noalloc(B, op, n, s, nu, length, dt, u, K)
    assert np.abs(got - want).max() <= TOL * np.abs(want).max(), (op, n, s)
    ref_norm = np.linalg.norm(want)
    assert abs(fnorm - ref_norm) <= TOL * ref_norm, (op, n, s, fnorm, ref_norm)
    if against_regular:
        reg = _regular(B, op, n, s, nu, length, dt, u, K)
        assert np.abs(got - reg).max() <= TOL * np.abs(reg).max(), (op, n, s)


@pytest.mark.parametrize("op,s,length", [("burgers2d", 3, 1.0), ("vsf", 5, 2 * math.pi)])
def test_noalloc_larger_then_smaller_grid(B, op, s, length):
    """128^2 (64 partial slots) and then 32^2 (4 slots) on the shared array."""
    _check(B, op, 128, s, length, seed=1)
    _check(B, op, 32, s, length, seed=2)


@pytest.mark.parametrize("op,n,s", [("burgers1d", 256, 2), ("diffusion1d", 512, 4)])
def test_noalloc_1d_operators_twice(B, op, n, s):
    _check(B, op, n, s, 1.0, seed=3)
    _check(B, op, n, s, 1.0, seed=4)


@pytest.mark.parametrize("op,s,length", [("burgers2d", 2, 1.0), ("vsf", 2, 2 * math.pi)])
def test_noalloc_at_its_scratch_limit(B, op, s, length):
    """1024^2 points: exactly 4096 blocks, every slot of the array in use."""
    _check(B, op, 1024, s, length, seed=5, against_regular=False)


def test_noalloc_rejects_grids_beyond_its_scratch(B):
    dev = torch.device("cuda", 0)
    tiny = torch.zeros(4, dtype=torch.float64, device=dev)
    A = B.irk_tableau(2)["A"]
    with pytest.raises(B.IrkError) as ei:
        B.irk_stage_residual_noalloc("burgers2d", 2048, 1.0, 0.01, 2, A, 1e-3,
                                     tiny, tiny, tiny, tiny)
    assert ei.value.status == B.IRK_ERR_NOMEM


def test_noalloc_rejects_memory_of_another_device_before_any_launch(B):
    """The library checks that each buffer is memory of the current device.
    Host memory stands in for a buffer the kernels cannot reach (this box has
    one GPU); the call must return IRK_ERR_INVALID and launch nothing."""
    n, s = 32, 2
    dev = torch.device("cuda", 0)
    A = np.ascontiguousarray(B.irk_tableau(s)["A"])
    u = torch.zeros((2, n, n), dtype=torch.float64, device=dev)
    K = torch.zeros((s, 2, n, n), dtype=torch.float64, device=dev)
    F = torch.full((s, 2, n, n), 7.0, dtype=torch.float64, device=dev)
    fnorm = torch.full((1,), 7.0, dtype=torch.float64, device=dev)
    host = np.zeros(s * 2 * n * n)
    torch.cuda.synchronize(dev)
    vp = C.c_void_p
    for bad in range(4):
        ptrs = [vp(x.data_ptr()) for x in (u, K, F, fnorm)]
        ptrs[bad] = vp(host.ctypes.data)
        st = B.LIB.irk_stage_residual_noalloc(B.IRK_OP_BURGERS_2D, n, 1.0, 0.01, s,
                                              A.ctypes.data, 1e-3, *ptrs, None)
        assert st == B.IRK_ERR_INVALID, (bad, st)
    torch.cuda.synchronize(dev)
    assert bool((F == 7.0).all()) and float(fnorm.item()) == 7.0
    assert np.all(host == 0.0)
