"""The full-size workloads over their full step counts, against the oracle.

2D viscous Burgers 512^2 (Gauss s = 2 and 3, dt = 2e-3, 50 steps) and the
vorticity-streamfunction DAE 1024^2 (Gauss s = 5, dt = 5e-3, 20 steps), run on
the GPU exactly as the benchmark runs them (one IRK step per call, the
extrapolated Newton start, whole-step CUDA graphs).  Every step is checked
against the oracle's definition of the result (Sec. 1.1 Eq. stages/update;
Sec. 6 Eq. dae_stage):

* the GPU's stage vectors k_i, put into the oracle's stage residual about the
  GPU's u_n, satisfy ||F|| <= 2e-10 ||F(k=0)|| (Newton tolerance 1e-10 plus
  rounding of the evaluation),
* u_{n+1} = u_n + dt sum_i b_i k_i to rounding,
* ||u_{n+1}|| agrees with the oracle's trajectory to 1e-9,

and after the last step the state matches the oracle's to 1e-8 relative L2.
The oracle's trajectories come from tests/golden/make_trajectories.py, which
calls only `oracle/`.  The mixed-precision V-cycles of the DAE (FP32, and
BF16 storage with FP32 arithmetic) are compared with the oracle's first step.
"""
import math
import os

import numpy as np
import pytest

import workloads
from oracle import irk as orc
from oracle import tableau as tab
from oracle import vsf as ovsf
from oracle.operators import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP_TOL = 1e-9
RUN_TOL = 1e-8
RESID_TOL = 2e-10
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def golden(case):
    path = os.path.join(GOLDEN, f"traj_{case}.npz")
    if case.startswith("vsf") and not os.path.exists(path):
        # the oracle needs hours for this trajectory (GMRES on 5 x 1024^2
        # unknowns, 20 steps); until its file is written the DAE cases wait
        pytest.skip(f"{path} not written yet (tests/golden/make_trajectories.py {case})")
    assert os.path.exists(path), f"{path} missing: run tests/golden/make_trajectories.py {case}"
    return dict(np.load(path))


def setup(case):
    g = golden(case)
    n, nu, dt, s, seed = int(g["n"]), float(g["nu"]), float(g["dt"]), int(g["stages"]), int(g["seed"])
    if case.startswith("vsf"):
        p = Problem("vsf", n, nu, 2 * math.pi)
        u0 = ovsf.initial_state(workloads.double_shear_layer_vorticity(n, seed=seed), p.h)
        kw = dict(op="vsf", length=2 * math.pi)
    else:
        p = Problem("burgers2d", n, nu, 1.0)
        u0 = workloads.random_fourier_2d(n, seed=seed)
        kw = dict(op="burgers2d", length=1.0)
    return g, p, u0, dict(n=n, stages=s, nu=nu, **kw), dt


def oracle_state(case, omega_or_u, h):
    if case.startswith("vsf"):
        return np.stack([omega_or_u, ovsf.poisson_solve(omega_or_u, h)])
    return omega_or_u


@pytest.mark.parametrize("case", ["burgers2d_512_gauss2", "burgers2d_512_gauss3", "vsf_1024_gauss5"])
def test_full_run_matches_oracle_trajectory(B, case):
    g, p, u0, kw, dt = setup(case)
    s = kw["stages"]
    A, b, c = tab.gauss(s)
    nsteps = int(g["nsteps"])
    worst_res, worst_norm, its = 0.0, 0.0, []
    with B.IrkSolver(u0.copy(), **kw) as sol:
        sol.set_state(u0)  # the oracle's consistent psi_0 for the DAE
        u_n = u0.copy()
        t = 0.0
        for k in range(nsteps):
            st = sol.step(t, dt, 1)
            its.append((st.newton_its, st.krylov_its))
            K = sol.stages()
            u1 = sol.state()
            F = orc.stage_residual(p, u_n, K, t, dt, A, c)
            F0 = orc.stage_residual(p, u_n, np.zeros_like(K), t, dt, A, c)
            r = np.linalg.norm(F) / np.linalg.norm(F0)
            worst_res = max(worst_res, r)
            assert r <= RESID_TOL, (case, k, r, st.as_dict())
            assert rel(u1, u_n + dt * np.tensordot(b, K, axes=(0, 0))) <= 1e-14, (case, k)
            dn = abs(np.linalg.norm(u1) - g["norms"][k + 1]) / g["norms"][k + 1]
            worst_norm = max(worst_norm, dn)
            assert dn <= STEP_TOL, (case, k, dn)
            u_n = u1
            t += dt
    want = oracle_state(case, g["u_final"], p.h)
    err = rel(u_n, want)
    print(f"{case}: {nsteps} steps, rel L2 {err:.2e}, worst stage residual {worst_res:.2e}, "
          f"worst norm drift {worst_norm:.2e}, (newton, krylov) per step {its[:3]}...")
    assert err <= RUN_TOL, (case, err)


@pytest.mark.parametrize("prec", [1, 2])
def test_vsf_1024_reduced_precision_vcycles_first_step(B, prec):
    """Config [2] with the V-cycle in FP32 (1) and in BF16 storage with FP32
    arithmetic (2); the Newton residual, stage update and Gram-Schmidt stay
    FP64, so the flexible outer iteration reaches the oracle's fixed point."""
    case = "vsf_1024_gauss5"
    g, p, u0, kw, dt = setup(case)
    with B.IrkSolver(u0.copy(), mg_precision=prec, **kw) as sol:
        sol.set_state(u0)
        st = sol.step(0.0, dt, 1)
        u1 = sol.state()
    err = rel(u1, oracle_state(case, g["u_step1"], p.h))
    print(f"vsf 1024 mg_precision {prec}: rel L2 {err:.2e}, {st.as_dict()}")
    assert err <= STEP_TOL, (prec, err, st.as_dict())
    assert st.final_rel_res <= 1e-10
