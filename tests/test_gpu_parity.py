"""CUDA path vs the FP64 oracle, through the C ABI.

Tolerances (spec contract): per step, starting from the oracle's u_n,
the GPU u_{n+1} matches the oracle within 1e-9 relative L2 at Newton relative
residual 1e-10; over a full run within 1e-8.  Operator kernels (residual,
Jacobian-vector product) are compared element by element at 1e-12 relative
to the largest entry (differences are rounding order only).
"""
import math

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


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_01776_gb300 import build
    build.build()
    from paper_2101_01776_gb300 import binding
    return binding


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def make_problem(op, n, nu, s):
    length = 2 * math.pi if op == "vsf" else 1.0
    return Problem(op, n, nu, length), length


def initial(op, n, seed):
    if op == "burgers1d" or op == "diffusion1d":
        return workloads.burgers1d_initial(n, seed=seed)[None]
    if op == "burgers2d":
        return workloads.random_fourier_2d(n, seed=seed)
    w0 = workloads.double_shear_layer_vorticity(n, seed=seed)
    return ovsf.initial_state(w0, 2 * math.pi / n)


def oracle_step(p, s, u, t, dt, family="gauss"):
    if p.op == "vsf":
        return ovsf.reduced_step(p, s, u, t, dt, family=family)
    linear = "direct" if p.size * s <= 40000 else "gmres"
    return orc.step(p, s, u, t, dt, linear=linear, family=family)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("op,n,s", [("diffusion1d", 64, 2), ("burgers1d", 64, 2), ("burgers1d", 64, 5),
                                    ("burgers2d", 32, 2), ("burgers2d", 16, 3), ("vsf", 32, 3),
                                    ("vsf", 16, 5)])
def test_stage_residual_matches_oracle(B, op, n, s):
    nu = 0.013
    p, length = make_problem(op, n, nu, s)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(p.shape)
    K = rng.standard_normal((s,) + p.shape)
    dt, t = 3e-3, 0.25
    A, b, c = tab.gauss(s)
    want = orc.stage_residual(p, u, K, t, dt, A, c)
    with B.IrkSolver(u, op=op, n=n, stages=s, nu=nu, length=length) as sol:
        sol.set_state(u)
        got = B.irk_stage_residual(sol.h, t, dt, K, np.empty_like(K))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_stage_residual_with_manufactured_forcing(B):
    n, s, nu = 64, 3, 0.02
    p = Problem("burgers1d", n, nu, forcing=1)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(p.shape)
    K = rng.standard_normal((s,) + p.shape)
    A, b, c = tab.gauss(s)
    want = orc.stage_residual(p, u, K, 0.7, 0.05, A, c)
    with B.IrkSolver(u, op="burgers1d", n=n, stages=s, nu=nu, forcing=1) as sol:
        got = B.irk_stage_residual(sol.h, 0.7, 0.05, K, np.empty_like(K))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("op,n,s", [("burgers1d", 64, 3), ("burgers2d", 16, 2), ("vsf", 16, 3)])
def test_stage_jacobian_matches_oracle(B, op, n, s):
    nu = 0.02
    p, length = make_problem(op, n, nu, s)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(p.shape)
    K = rng.standard_normal((s,) + p.shape)
    V = rng.standard_normal((s,) + p.shape)
    dt = 4e-3
    A, _, _ = tab.gauss(s)
    want = (orc.newton_matrix(p, u, K, dt, A) @ V.ravel()).reshape(V.shape)
    with B.IrkSolver(u, op=op, n=n, stages=s, nu=nu, length=length) as sol:
        sol.set_state(u)
        got = B.irk_stage_jacobian_apply(sol.h, dt, K, V, np.empty_like(V))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


# ---------------------------------------------------------------------------
def run_parity(B, op, n, s, nu, dt, nsteps, seed=0, device_buffers=False, **cfg):
    p, length = make_problem(op, n, nu, s)
    u0 = initial(op, n, seed)
    family = cfg.get("family", "gauss")
    per_step, infos = [], []
    u_ref = u0.copy()
    with B.IrkSolver(u0 if op != "vsf" else u0.copy(), op=op, n=n, stages=s, nu=nu,
                     length=length, **cfg) as sol:
        # per step, restarting from the oracle's state
        t = 0.0
        for k in range(nsteps):
            sol.set_state(u_ref)
            st = sol.step(t, dt, 1)
            infos.append(st.as_dict())
            u_next, _, _ = oracle_step(p, s, u_ref, t, dt, family)
            per_step.append(rel(sol.state(), u_next))
            u_ref = u_next
            t += dt
        # whole run from u0
        start = u0 if op != "vsf" else initial(op, n, seed)
        if device_buffers:
            d = torch.from_numpy(start.copy()).cuda()
            sol.set_state(d)
        else:
            sol.set_state(start)
        sol.step(0.0, dt, nsteps)
        whole = rel(sol.state(), u_ref)
    return per_step, whole, infos


def test_config0_burgers1d_n256_gauss2_10_steps(B):
    """1D viscous Burgers, N=256, nu=0.01, Gauss s=2, dt=1e-3, 10 steps."""
    per_step, whole, infos = run_parity(B, "burgers1d", 256, 2, 0.01, 1e-3, 10, seed=0)
    assert max(per_step) <= STEP_TOL, per_step
    assert whole <= RUN_TOL, whole
    assert all(i["final_rel_res"] <= 1e-10 for i in infos)
    # s = 2 with Newton-like(3) is exact Newton: a few iterations per step
    assert all(i["newton_its"] <= 4 for i in infos), infos


@pytest.mark.parametrize("s", [1, 3, 4, 5])
def test_burgers1d_all_stage_counts(B, s):
    per_step, whole, _ = run_parity(B, "burgers1d", 128, s, 0.01, 2e-3, 3, seed=1)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole)


@pytest.mark.parametrize("n,s", [(32, 2), (64, 2), (64, 3), (16, 5)])
def test_burgers2d_parity(B, n, s):
    per_step, whole, infos = run_parity(B, "burgers2d", n, s, 5e-3, 2e-3, 3, seed=1)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)


@pytest.mark.parametrize("n,s", [(32, 2), (32, 3), (16, 5)])
def test_vsf_parity(B, n, s):
    per_step, whole, infos = run_parity(B, "vsf", n, s, 1e-3, 5e-3, 2, seed=2)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_preconditioner_same_result(B, prec):
    """FP32 / BF16-stored V-cycles change Krylov counts, not the fixed point."""
    per_step, whole, infos = run_parity(B, "burgers2d", 64, 3, 5e-3, 2e-3, 2, seed=3,
                                        mg_precision=prec)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole)


@pytest.mark.parametrize("op,n,s,prec", [("burgers2d", 64, 2, 1), ("burgers2d", 32, 2, 2),
                                         ("vsf", 64, 2, 1), ("vsf", 32, 3, 2), ("burgers1d", 128, 2, 1)])
def test_mixed_precision_fine_level_reads_fp64(B, op, n, s, prec):
    """Reduced-precision V-cycles whose finest level reads the FP64 input and
    writes the FP64 output directly (and, for 2-stage Gauss and the VSF
    rows, the L_P coupling right-hand side with it) reach the oracle's fixed
    point; the V-cycle then launches no conversion kernels."""
    nu, dt = {"burgers1d": (0.01, 2e-3), "burgers2d": (5e-3, 2e-3), "vsf": (1e-3, 5e-3)}[op]
    per_step, whole, infos = run_parity(B, op, n, s, nu, dt, 2, seed=12, mg_precision=prec)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)
    if op == "burgers2d":
        u0 = initial(op, n, 12)
        with B.IrkSolver(u0, op=op, n=n, stages=s, nu=nu, mg_precision=prec, profile=1) as sol:
            sol.step(0.0, dt, 1)
            names = {k["name"] for k in B.irk_kernel_stats(sol.h)}
        assert "mg_convert" not in names, names


@pytest.mark.parametrize("kw", [dict(gamma_mode=1), dict(nonlinear_variant=2),
                                dict(krylov_restart=3), dict(mg_levels=2),
                                dict(mg_coarse_smoother=2), dict(mg_coarse_smoother=1),
                                dict(mg_shifted_sweeps=0), dict(mg_tile_rows=8),
                                dict(mg_tile_rows=16, mg_precision=1), dict(nonlinear_variant=3)])
def test_solver_variants_reach_same_fixed_point(B, kw):
    per_step, whole, _ = run_parity(B, "burgers2d", 32, 3, 5e-3, 2e-3, 2, seed=4, **kw)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (kw, per_step, whole)


@pytest.mark.parametrize("family,s", [("radau", 1), ("radau", 2), ("radau", 3), ("radau", 5),
                                      ("lobatto", 2), ("lobatto", 3), ("lobatto", 4)])
def test_radau_lobatto_burgers1d_parity(B, family, s):
    """Radau IIA and Lobatto IIIC tableaux (Table 1) through the same solver."""
    per_step, whole, infos = run_parity(B, "burgers1d", 128, s, 0.01, 2e-3, 3, seed=1,
                                        family=family)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)


@pytest.mark.parametrize("op,n,family,s", [("burgers2d", 32, "radau", 3), ("burgers2d", 32, "lobatto", 2),
                                           ("vsf", 32, "radau", 2), ("vsf", 16, "lobatto", 3)])
def test_radau_lobatto_2d_parity(B, op, n, family, s):
    nu, dt = (5e-3, 2e-3) if op == "burgers2d" else (1e-3, 5e-3)
    per_step, whole, infos = run_parity(B, op, n, s, nu, dt, 2, seed=2, family=family)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)


@pytest.mark.parametrize("op,n,s,family", [("burgers1d", 128, 2, "gauss"), ("burgers1d", 128, 5, "gauss"),
                                           ("burgers2d", 32, 3, "gauss"), ("burgers2d", 32, 4, "radau"),
                                           ("vsf", 32, 3, "gauss")])
def test_eigenvector_basis_reaches_same_fixed_point(B, op, n, s, family):
    """The real eigenvector basis of A0^{-1} (non-orthogonal T) in place of the
    Schur basis: the transform changes the iteration, not the solution."""
    nu, dt = {"burgers1d": (0.01, 2e-3), "burgers2d": (5e-3, 2e-3), "vsf": (1e-3, 5e-3)}[op]
    per_step, whole, infos = run_parity(B, op, n, s, nu, dt, 2, seed=6, basis=1, family=family)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)


@pytest.mark.parametrize("variant", [0, 1, 4])
@pytest.mark.parametrize("op,n,s", [("burgers2d", 32, 3), ("burgers1d", 128, 4), ("vsf", 32, 3)])
def test_nonlinear_variants_0_1_4(B, variant, op, n, s):
    """Simplified Newton (0), lumped block diagonal (1) and exact Newton (4, outer
    FGMRES on the true Jacobian) reach the same fixed point (Sec. 3.2)."""
    nu, dt = {"burgers1d": (0.01, 2e-3), "burgers2d": (5e-3, 2e-3), "vsf": (1e-3, 5e-3)}[op]
    per_step, whole, infos = run_parity(B, op, n, s, nu, dt, 2, seed=7, nonlinear_variant=variant)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)
    if variant == 4:
        assert all(i["outer_its"] > 0 for i in infos), infos
    else:
        assert all(i["outer_its"] == 0 for i in infos), infos


def test_exact_newton_converges_quadratically(B):
    """Variant 4 is Newton on the true stage Jacobian: for s = 4 it needs no more
    iterations than the block upper triangular variant 3, and at most 4 here."""
    its = {}
    for v in (3, 4):
        _, _, infos = run_parity(B, "burgers2d", 32, 4, 5e-3, 4e-3, 2, seed=8, nonlinear_variant=v)
        its[v] = [i["newton_its"] for i in infos]
    assert all(a <= b for a, b in zip(its[4], its[3])), its
    assert max(its[4]) <= 4, its


@pytest.mark.parametrize("family,s,k", [("radau", 3, 2), ("lobatto", 3, 1), ("radau", 1, 0)])
def test_linear_diffusion_pade_radau_lobatto(B, family, s, k):
    """Per Fourier mode, one step multiplies by the (k, s) Pade approximant of
    exp(dt lambda_m): k = s-1 for Radau IIA, s-2 for Lobatto IIIC."""
    n, nu, dt = 64, 0.05, 0.004
    u0 = np.random.default_rng(s + 10).standard_normal((1, n))
    with B.IrkSolver(u0, op="diffusion1d", n=n, stages=s, nu=nu, family=family) as sol:
        sol.step(0.0, dt, 1)
        u1 = sol.state()
    f = math.factorial
    m = np.arange(n)
    z = -dt * (4 * nu * n * n) * np.sin(np.pi * m / n) ** 2
    P = sum(f(k + s - i) * f(k) / (f(k + s) * f(i) * f(k - i)) * z ** i for i in range(k + 1))
    Q = sum(f(k + s - i) * f(s) / (f(k + s) * f(i) * f(s - i)) * (-z) ** i for i in range(s + 1))
    want = np.real(np.fft.ifft(P / Q * np.fft.fft(u0[0])))
    assert rel(u1[0], want) <= 1e-9


@pytest.mark.parametrize("seq,guess", [(1, 2), (0, 2), (1, 0)])
@pytest.mark.parametrize("op,n,s", [("burgers1d", 128, 1), ("burgers1d", 128, 2), ("burgers1d", 128, 3),
                                    ("burgers1d", 128, 5), ("burgers2d", 32, 3), ("burgers2d", 16, 5),
                                    ("vsf", 32, 2), ("vsf", 16, 3)])
def test_sdirk_parity(B, op, n, s, seq, guess):
    """SDIRK, the diagonally implicit comparison of Sec. 7, stage by stage
    (seq = 1: every stage its own Newton loop on the single-stage solver) and
    coupled (seq = 0: Algorithm 1 over the stage system, whose transformed
    Jacobian is exactly block upper triangular): both reach the oracle's
    solution of the full stage equations."""
    nu, dt = {"burgers1d": (0.01, 2e-3), "burgers2d": (5e-3, 2e-3), "vsf": (1e-3, 5e-3)}[op]
    per_step, whole, infos = run_parity(B, op, n, s, nu, dt, 2, seed=9, family="sdirk",
                                        dirk_sequential=seq, initial_guess=guess)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)
    # 1x1 blocks only: one preconditioner application per Krylov iteration
    assert all(i["prec_apps"] == i["krylov_its"] > 0 for i in infos), infos
    if seq:
        # every stage runs at least one Newton iteration of its own
        assert all(i["newton_its"] >= s for i in infos), infos
    if op == "vsf":
        # one stream function V-cycle per preconditioner application
        assert all(i["poisson_vcycles"] == i["prec_apps"] for i in infos), infos


@pytest.mark.parametrize("s", [1, 2, 3, 5])
def test_sdirk_linear_diffusion_stability_function(B, s):
    """Per Fourier mode one SDIRK step multiplies by R(z) = 1 + z b^T (I - z A)^{-1} 1,
    z = dt lambda_m (the tableau's stability function)."""
    n, nu, dt = 64, 0.05, 0.004
    u0 = np.random.default_rng(s + 20).standard_normal((1, n))
    with B.IrkSolver(u0, op="diffusion1d", n=n, stages=s, nu=nu, family="sdirk") as sol:
        sol.step(0.0, dt, 1)
        u1 = sol.state()
    A, b, _ = tab.sdirk(s)
    m = np.arange(n)
    z = -dt * (4 * nu * n * n) * np.sin(np.pi * m / n) ** 2
    R = np.array([1.0 + zz * (b @ np.linalg.solve(np.eye(s) - zz * A, np.ones(s))) for zz in z])
    want = np.real(np.fft.ifft(R * np.fft.fft(u0[0])))
    assert rel(u1[0], want) <= 1e-9


def test_sdirk_stage_by_stage_profile_and_kernel_stats(B):
    """Profiled stage-by-stage SDIRK: the stage solver's kernel classes are
    reported through the outer handle."""
    u0 = initial("burgers2d", 32, 3)
    with B.IrkSolver(u0, op="burgers2d", n=32, stages=3, nu=5e-3, family="sdirk", profile=1) as sol:
        st = sol.step(0.0, 2e-3, 2).as_dict()
        ks = {k["name"]: k for k in B.irk_kernel_stats(sol.h)}
    assert st["steps"] == 2 and st["newton_its"] >= 6, st
    for name in ("residual", "stage_op", "mg_smooth"):
        assert name in ks and ks[name]["launches"] > 0 and ks[name]["ms"] > 0, ks.keys()


@pytest.mark.parametrize("n,s,family,prec", [(32, 2, "gauss", 0), (32, 3, "gauss", 0), (16, 5, "gauss", 0),
                                              (32, 1, "gauss", 0), (16, 3, "sdirk", 0), (32, 2, "radau", 0),
                                              (32, 3, "gauss", 1), (32, 2, "gauss", 2)])
def test_vsf_block_triangular_forward_solve_parity(B, n, s, family, prec):
    """Eq. vsf-system-2 (dae_solver = 1): the block forward solve of the
    reordered Picard system (FGMRES on the omega block with the omega part of
    L_P, then one MG-preconditioned Poisson FGMRES per stream function row)
    reaches the oracle's fixed point; the stream function V-cycles are
    counted apart from the omega V-cycles."""
    per_step, whole, infos = run_parity(B, "vsf", n, s, 1e-3, 5e-3, 2, seed=2, dae_solver=1,
                                        family=family, mg_precision=prec)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)
    for i in infos:
        omega = i["vcycles"] - i["poisson_vcycles"]
        assert i["poisson_vcycles"] > 0 and omega == i["prec_apps"] > 0, i


def test_vsf_forward_solve_counts_against_eq_vsf_system_1(B):
    """Both DAE solvers on the same step: Eq. vsf-system-1 applies one omega
    and one psi V-cycle per preconditioner application; the forward solve
    spends its psi V-cycles in the Poisson solves instead (the paper's
    comparison of the two, Table dsl-iters, reports both counts)."""
    n, s = 32, 3
    u0 = initial("vsf", n, 5)
    out = {}
    for ds in (0, 1):
        with B.IrkSolver(u0.copy(), op="vsf", n=n, stages=s, nu=1e-3, length=2 * math.pi,
                         dae_solver=ds) as sol:
            out[ds] = (sol.step(0.0, 5e-3, 2).as_dict(), sol.state())
    assert rel(out[1][1], out[0][1]) <= 2 * STEP_TOL
    a, b = out[0][0], out[1][0]
    assert a["poisson_vcycles"] == a["prec_apps"], a
    assert b["poisson_vcycles"] > 0 and b["vcycles"] - b["poisson_vcycles"] == b["prec_apps"], b


def test_device_buffers_and_minimum_grid(B):
    per_step, whole, _ = run_parity(B, "burgers2d", 8, 2, 5e-3, 2e-3, 2, seed=5, device_buffers=True)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_linear_diffusion_pade_per_mode(B, s):
    n, nu, dt = 64, 0.05, 0.004
    u0 = np.random.default_rng(s).standard_normal((1, n))
    with B.IrkSolver(u0, op="diffusion1d", n=n, stages=s, nu=nu) as sol:
        sol.step(0.0, dt, 1)
        u1 = sol.state()
    coef = [math.factorial(2 * s - j) * math.factorial(s)
            / (math.factorial(2 * s) * math.factorial(j) * math.factorial(s - j)) for j in range(s + 1)]
    m = np.arange(n)
    z = -dt * (4 * nu * n * n) * np.sin(np.pi * m / n) ** 2
    R = np.polyval(coef[::-1], z) / np.polyval(coef[::-1], -z)
    want = np.real(np.fft.ifft(R * np.fft.fft(u0[0])))
    assert rel(u1[0], want) <= 1e-9


# ---------------------------------------------------------------------------
def test_full_size_burgers2d_512_one_step(B):
    """2D Burgers 512^2, Gauss s=2, dt=2e-3 (the benchmark workload): the GPU
    stages satisfy the oracle's stage equations to the Newton tolerance, the
    update matches Eq. update, and u_{n+1} matches the oracle's GMRES variant."""
    n, s, nu, dt = 512, 2, 5e-3, 2e-3
    p = Problem("burgers2d", n, nu)
    u0 = workloads.random_fourier_2d(n, seed=1)
    with B.IrkSolver(u0, op="burgers2d", n=n, stages=s, nu=nu) as sol:
        st = sol.step(0.0, dt, 1)
        u1 = sol.state()
        K = sol.stages()
    A, b, c = tab.gauss(s)
    F = orc.stage_residual(p, u0, K, 0.0, dt, A, c)
    F0 = orc.stage_residual(p, u0, np.zeros_like(K), 0.0, dt, A, c)
    assert np.linalg.norm(F) <= 2e-10 * np.linalg.norm(F0)
    assert rel(u1, u0 + dt * np.tensordot(b, K, axes=(0, 0))) <= 1e-14
    ref, _, _ = orc.step(p, s, u0, 0.0, dt, linear="gmres")
    assert rel(u1, ref) <= STEP_TOL


# ---------------------------------------------------------------------------
def test_edge_cases(B):
    n = 64
    zero = np.zeros((1, n))
    with B.IrkSolver(zero, op="burgers1d", n=n, stages=2, nu=0.01) as sol:
        st = sol.step(0.0, 1e-3, 3)              # F(0) = 0: converged at k = 0
        assert st.steps == 3 and st.newton_its == 0
        assert np.all(sol.state() == 0)
        st = sol.step(0.0, 1e-3, 0)              # nsteps = 0 is a no-op
        assert st.steps == 0
        with pytest.raises(B.IrkError):
            sol.step(0.0, -1e-3, 1)
        with pytest.raises(B.IrkError):
            sol.step(0.0, float("nan"), 1)


def test_failed_step_leaves_state_untouched(B):
    n = 64
    u0 = workloads.burgers1d_initial(n, seed=0)[None]
    with B.IrkSolver(u0, op="burgers1d", n=n, stages=2, nu=0.01, newton_maxit=1) as sol:
        before = sol.state().copy()
        with pytest.raises(B.IrkError) as ei:
            sol.step(0.0, 1e-2, 1)
        assert ei.value.status == B.IRK_ERR_NEWTON_MAXIT
        np.testing.assert_array_equal(sol.state(), before)
    bad = u0.copy()
    bad[0, 3] = np.nan
    with B.IrkSolver(bad, op="burgers1d", n=n, stages=2, nu=0.01) as sol:
        with pytest.raises(B.IrkError) as ei:
            sol.step(0.0, 1e-3, 1)
        assert ei.value.status == B.IRK_ERR_NEWTON_DIVERGED


def test_checkpoint_resume_and_determinism_bit_equal(B):
    n, s = 64, 3
    u0 = workloads.random_fourier_2d(n, seed=7)
    kw = dict(op="burgers2d", n=n, stages=s, nu=5e-3)
    with B.IrkSolver(u0, **kw) as a:
        a.step(0.0, 2e-3, 4)
        full = a.state().copy()
        a.set_state(u0)
        a.step(0.0, 2e-3, 4)
        again = a.state().copy()
    with B.IrkSolver(u0, **kw) as b:
        b.step(0.0, 2e-3, 2)
        ck = b.state().copy()
        ck_stages = b.stages().copy()  # the warm-start guess of the next step
    with B.IrkSolver(ck, **kw) as c:
        c.set_stages(ck_stages)
        c.step(2 * 2e-3, 2e-3, 2)
        resumed = c.state().copy()
    np.testing.assert_array_equal(full, again)
    np.testing.assert_array_equal(full, resumed)


@pytest.mark.parametrize("guess", [0, 1, 2])
def test_initial_guess_reaches_the_same_fixed_point(B, guess):
    """Newton from zero stages, from the previous step's stages or from their
    extrapolation along the collocation polynomial: the same stage equations,
    the same tolerance (relative to ||F(k=0)||)."""
    per_step, whole, infos = run_parity(B, "burgers2d", 64, 2, 5e-3, 2e-3, 3, seed=6,
                                        initial_guess=guess)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)


@pytest.mark.parametrize("graphs,family,s", [(1, "gauss", 2), (0, "gauss", 3), (1, "sdirk", 2),
                                              (1, "radau", 3)])
def test_bad_warm_start_restarts_from_zero(B, graphs, family, s):
    """A warm start whose residual exceeds that of zero stages (here: stages
    set to large noise) is rejected and the step restarts from zero, from the
    saved state: it still reaches the oracle's solution (graph path, host
    path, and the stage solver of stage-by-stage SDIRK)."""
    op, n, nu, dt = "burgers2d", 32, 5e-3, 2e-3
    p, _ = make_problem(op, n, nu, s)
    u0 = initial(op, n, 13)
    with B.IrkSolver(u0, op=op, n=n, stages=s, nu=nu, family=family, use_graphs=graphs) as sol:
        bad = 1e3 * np.random.default_rng(0).standard_normal((s,) + u0.shape)
        sol.set_stages(np.ascontiguousarray(bad))
        st = sol.step(0.0, dt, 1).as_dict()
        got = sol.state()
    want, _, _ = oracle_step(p, s, u0, 0.0, dt, family)
    assert rel(got, want) <= STEP_TOL, (rel(got, want), st)
    assert st["final_rel_res"] <= 1e-10, st


@pytest.mark.parametrize("op,n,s,family", [("burgers2d", 64, 3, "gauss"), ("vsf", 64, 5, "gauss"),
                                           ("burgers2d", 64, 3, "radau"), ("burgers1d", 256, 4, "gauss")])
def test_extrapolated_guess_saves_iterations(B, op, n, s, family):
    """Over a smooth trajectory the extrapolated starting value (guess 2) needs
    no more Krylov iterations than the previous stages (guess 1), and the two
    runs agree to the Newton tolerance; a step after a change of dt and a
    reset state still converge."""
    nu, dt, length = {"burgers1d": (0.01, 2e-3, 1.0), "burgers2d": (5e-3, 2e-3, 1.0),
                      "vsf": (1e-3, 5e-3, 2 * math.pi)}[op]
    u0 = initial(op, n, 8)
    kry, out = {}, {}
    for guess in (1, 2):
        with B.IrkSolver(u0.copy(), op=op, n=n, stages=s, nu=nu, length=length, family=family,
                         initial_guess=guess) as sol:
            sol.step(0.0, dt, 2)
            st = sol.step(2 * dt, dt, 4).as_dict()
            kry[guess] = st["krylov_its"]
            out[guess] = sol.state().copy()
            st2 = sol.step(6 * dt, 0.5 * dt, 2).as_dict()  # dt change: ratio 1/2
            sol.set_state(out[guess])
            st3 = sol.step(6 * dt, dt, 1).as_dict()  # reset: zero stages
            assert st2["steps"] == 2 and st3["steps"] == 1
    assert kry[2] <= kry[1], kry
    assert rel(out[2], out[1]) <= 1e-9, rel(out[2], out[1])


def test_graph_path_matches_host_driven_path(B):
    """The CUDA-graph path (L_P replay, FGMRES loop in a WHILE node with the
    Arnoldi/Givens step on the device) reaches the same iterates as the
    host-driven loop: same Krylov counts, states equal to rounding."""
    n, s = 64, 3
    u0 = workloads.random_fourier_2d(n, seed=9)
    stream = torch.cuda.Stream()
    outs = []
    for graphs in (0, 1):
        with B.IrkSolver(torch.from_numpy(u0).cuda(), stream=stream, op="burgers2d", n=n,
                         stages=s, nu=5e-3, use_graphs=graphs) as sol:
            st = sol.step(0.0, 2e-3, 3)
            outs.append((sol.state().copy(), st.krylov_its, st.vcycles))
    assert rel(outs[1][0], outs[0][0]) <= 1e-12
    assert outs[0][1:] == outs[1][1:]


@pytest.mark.parametrize("op,n,s,prec,graphs", [("burgers2d", 64, 2, 0, 1), ("burgers2d", 64, 3, 1, 1),
                                               ("burgers2d", 128, 2, 2, 1), ("burgers2d", 64, 2, 0, 0),
                                               ("vsf", 64, 3, 0, 1), ("vsf", 64, 2, 1, 0)])
def test_fused_residual_restriction_is_bit_identical(B, op, n, s, prec, graphs):
    """The V-cycle's folded-pre-sweep residual and its restriction in one
    kernel (mg_fuse_transfer = 1) against the two separate kernels (2): the same
    operations in the same order, so the states are equal bit for bit and the
    Newton, Krylov and V-cycle counts agree (FP64, FP32 and BF16 storage;
    Burgers' precomputed and per-point coefficients; the VSF vorticity rows;
    graph and host-driven loops)."""
    nu = 5e-3 if op == "burgers2d" else 1e-3
    _, length = make_problem(op, n, nu, s)
    u0 = initial(op, n, seed=6)
    outs = []
    for fuse in (2, 1):
        with B.IrkSolver(u0.copy(), op=op, n=n, stages=s, nu=nu, length=length, mg_precision=prec,
                         use_graphs=graphs, mg_fuse_transfer=fuse) as sol:
            st = sol.step(0.0, 2e-3 if op == "burgers2d" else 5e-3, 3)
            outs.append((sol.state().copy(), st.newton_its, st.krylov_its, st.vcycles))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:] and outs[1][3] > 0


def test_vsf_medium_128_gauss5_parity(B):
    """Vorticity-streamfunction DAE, 128^2, Gauss s=5 (order 10), dt=5e-3, Re=1000."""
    per_step, whole, infos = run_parity(B, "vsf", 128, 5, 1e-3, 5e-3, 2, seed=2)
    assert max(per_step) <= STEP_TOL and whole <= RUN_TOL, (per_step, whole, infos)


def test_full_size_vsf_1024_gauss5_one_step(B):
    """Config [2] at full size (1024^2, s=5, dt=5e-3, Re=1000): the GPU stage
    vectors satisfy the oracle's DAE stage equations (Eq. dae_stage) to the
    Newton tolerance, the update matches Eq. update, the constraint -L psi =
    omega holds after the step and the mean of omega is conserved."""
    n, s, nu, dt = 1024, 5, 1e-3, 5e-3
    p = Problem("vsf", n, nu, 2 * math.pi)
    st0 = ovsf.initial_state(workloads.double_shear_layer_vorticity(n, seed=2), p.h)
    with B.IrkSolver(st0.copy(), op="vsf", n=n, stages=s, nu=nu, length=2 * math.pi) as sol:
        sol.set_state(st0)
        info = sol.step(0.0, dt, 1)
        u1 = sol.state()
        K = sol.stages()
    A, b, c = tab.gauss(s)
    F = orc.stage_residual(p, st0, K, 0.0, dt, A, c)
    F0 = orc.stage_residual(p, st0, np.zeros_like(K), 0.0, dt, A, c)
    assert np.linalg.norm(F) <= 2e-10 * np.linalg.norm(F0), info.as_dict()
    assert rel(u1, st0 + dt * np.tensordot(b, K, axes=(0, 0))) <= 1e-14
    g = p.N(u1)[1]
    assert np.abs(g).max() <= 1e-9 * np.abs(u1[0]).max()
    assert abs(u1[0].mean()) <= 1e-12 * np.abs(u1[0]).max()


def test_autotune_restores_state_and_keeps_parity(B):
    """irk_autotune times candidate V-cycle settings from the current state,
    restores state and stages, and keeps one of the candidates; stepping with
    the chosen settings still reaches the oracle's fixed point."""
    n, s, nu, dt = 64, 2, 5e-3, 2e-3
    p, length = make_problem("burgers2d", n, nu, s)
    u0 = initial("burgers2d", n, 9)
    with B.IrkSolver(u0, op="burgers2d", n=n, stages=s, nu=nu, length=length) as sol:
        sol.step(0.0, dt, 1)
        u1 = sol.state()
        k1 = sol.stages()
        chosen = B.irk_autotune(sol.h, dt, dt, 1)
        np.testing.assert_array_equal(sol.state(), u1)
        np.testing.assert_array_equal(sol.stages(), k1)
        got = B.irk_get_config(sol.h)
        assert got.mg_shifted_sweeps == chosen.mg_shifted_sweeps in (1, 2)
        assert got.mg_coarse_smoother == chosen.mg_coarse_smoother in (0, 2)
        assert got.mg_coarse_reduction in (2e-2, 5e-3)
        assert got.mg_tile_rows == chosen.mg_tile_rows in (0, 8, 16)
        assert got.mg_levels == chosen.mg_levels and got.mg_levels >= 0
        assert got.mg_fuse_transfer == chosen.mg_fuse_transfer in (0, 1, 2)
        sol.step(dt, dt, 1)
        u2 = sol.state()
    want, _, _ = oracle_step(p, s, u1, dt, dt)
    assert rel(u2, want) <= STEP_TOL


def test_set_state_keep_stages_keeps_the_guess(B):
    """irk_set_state_keep_stages replaces the state and keeps the stages as the
    Newton guess; irk_set_state zeroes them; both reach the oracle's u_{n+1}."""
    n, s, nu, dt = 32, 2, 5e-3, 2e-3
    p, length = make_problem("burgers2d", n, nu, s)
    u0 = initial("burgers2d", n, 10)
    with B.IrkSolver(u0, op="burgers2d", n=n, stages=s, nu=nu, length=length) as sol:
        sol.step(0.0, dt, 1)
        u1 = sol.state()
        k1 = sol.stages()
        assert np.abs(k1).max() > 0
        B.irk_set_state_keep_stages(sol.h, u1)
        np.testing.assert_array_equal(sol.stages(), k1)
        warm = sol.step(dt, dt, 1)
        u2w = sol.state()
        sol.set_state(u1)
        assert np.abs(sol.stages()).max() == 0
        cold = sol.step(dt, dt, 1)
        u2c = sol.state()
    want, _, _ = oracle_step(p, s, u1, dt, dt)
    assert rel(u2w, want) <= STEP_TOL and rel(u2c, want) <= STEP_TOL
    assert warm.newton_its <= cold.newton_its


def test_measured_alu_peaks_are_plausible(B):
    """irk_measure_alu_peak: FP64 FMA throughput within the derived ceiling
    (152 SMs x 2 DFMA/clk at up to 2070 MHz) and FP32 far above it."""
    fp64 = B.irk_measure_alu_peak(0)
    fp32 = B.irk_measure_alu_peak(1)
    derived64 = 152 * 2 * 2 * 2.070e9 / 1e12
    assert 0.3 * derived64 <= fp64 <= 1.05 * derived64, fp64
    assert fp32 >= 20 * fp64, (fp32, fp64)
    with pytest.raises(B.IrkError):
        B.irk_measure_alu_peak(2)


@pytest.mark.parametrize("s", [2, 3])
def test_profiled_path_runs_the_graph_kernels(B, s):
    """With per-kernel timing on (profile = 1) the block solves launch the
    kernels of the captured graph path one by one: the same iterates and
    Krylov counts as the graphs, and the timing classes of that path
    (fg_gs1, fg_gs2, fg_next) instead of the host-driven loop's."""
    n = 64
    u0 = workloads.random_fourier_2d(n, seed=14)
    outs = []
    for prof in (0, 1):
        with B.IrkSolver(u0, op="burgers2d", n=n, stages=s, nu=5e-3, profile=prof) as sol:
            st = sol.step(0.0, 2e-3, 3)
            outs.append((sol.state().copy(), st.krylov_its, st.newton_its))
            if prof:
                names = {k["name"]: k for k in B.irk_kernel_stats(sol.h)}
    assert rel(outs[1][0], outs[0][0]) <= 1e-12
    assert outs[0][1:] == outs[1][1:]
    for c in ("fg_gs1", "fg_gs2", "fg_next", "mg_smooth_tile", "stage_op"):
        assert names[c]["launches"] > 0 and names[c]["ms"] > 0, c
    assert names["fg_gs1"]["launches"] == names["fg_gs2"]["launches"] == outs[1][1]
    assert "gs_multi_dot" not in names or names["gs_multi_dot"]["launches"] == 0
