"""The allocation-free stage-residual entry point against the regular one.

irk_stage_residual_noalloc serves callers that cannot call cudaMalloc (a host
whose memory manager owns the device pool, a latency-critical loop that must
not synchronise the device through cudaMalloc/cudaFree, a fixed memory
budget).  Its scratch is a fixed file-scope device array shared by all calls,
so this file checks two calls in a row -- the second must not see anything
left behind by the first -- against irk_stage_residual, the entry point that
uses the handle's allocated buffers, at the same 1e-12 tolerance as the other
residual tests.  The file is named to be collected last.
"""
import numpy as np
import pytest

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


def _regular(B, op, n, s, nu, length, dt, u, K):
    with B.IrkSolver(u, op=op, n=n, stages=s, nu=nu, length=length) as sol:
        sol.set_state(u)
        return B.irk_stage_residual(sol.h, 0.0, dt, K, np.empty_like(K))


@pytest.mark.parametrize("op,n,s,length", [("burgers2d", 64, 3, 1.0), ("vsf", 32, 5, 2 * np.pi),
                                           ("burgers1d", 256, 2, 1.0)])
def test_noalloc_matches_regular_entry_twice(B, op, n, s, length):
    nu, dt = 0.011, 2.5e-3
    A = B.irk_tableau(s)["A"]
    shape = (2, n, n) if op in ("burgers2d", "vsf") else (1, n)
    rng = np.random.default_rng(123)
    dev = torch.device("cuda", 0)
    F = torch.empty((s,) + shape, dtype=torch.float64, device=dev)
    fnorm = torch.empty(1, dtype=torch.float64, device=dev)
    for call in range(2):
        u = rng.standard_normal(shape)
        K = rng.standard_normal((s,) + shape) * (1 + call)
        want = _regular(B, op, n, s, nu, length, dt, u, K)
        ud = torch.from_numpy(u).to(dev)
        Kd = torch.from_numpy(K).to(dev)
        F.fill_(float("nan"))
        fnorm.fill_(float("nan"))
        stream = torch.cuda.current_stream(dev)
        B.irk_stage_residual_noalloc(op, n, length, nu, s, A, dt, ud, Kd, F, fnorm, stream)
        torch.cuda.synchronize(dev)
        got = F.cpu().numpy()
        assert np.abs(got - want).max() <= TOL * np.abs(want).max(), (op, call)
        ref_norm = np.linalg.norm(want)
        assert abs(float(fnorm.item()) - ref_norm) <= TOL * ref_norm, (op, call)


def test_noalloc_rejects_grids_beyond_its_scratch(B):
    dev = torch.device("cuda", 0)
    tiny = torch.zeros(4, dtype=torch.float64, device=dev)
    A = B.irk_tableau(2)["A"]
    with pytest.raises(B.IrkError) as ei:
        B.irk_stage_residual_noalloc("burgers2d", 2048, 1.0, 0.01, 2, A, 1e-3,
                                     tiny, tiny, tiny, tiny)
    assert ei.value.status == B.IRK_ERR_NOMEM
