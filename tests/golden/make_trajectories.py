"""Write the oracle's full-size trajectories used by the full-size GPU parity tests.

    python tests/golden/make_trajectories.py [case ...]

Calls only `oracle/` (exact Newton at Newton relative residual 1e-10 plus one
extra iteration; SciPy GMRES to rtol 1e-13 on the assembled Jacobian for 2D
Burgers, the psi-eliminated FFT variant for the vorticity-streamfunction DAE)
and the seeded generators of `workloads/`.  Nothing here comes from the CUDA
path.  Each case writes `traj_<case>.npz` beside this file with

* `u_final`      the state after `nsteps` steps (VSF: omega only; the oracle's
                 psi is poisson_solve(omega), Sec. 6 constraint),
* `u_step1`      the state after the first step (VSF only, omega),
* `norms`        ||u_n||_2 for n = 0..nsteps,
* `newton_its`   oracle Newton iterations per step,
* `n, nu, dt, stages, seed` the workload, `nsteps` the steps written.

The file is rewritten after every step, so an interrupted run leaves a valid
shorter trajectory (its `nsteps` says how many steps it holds).

Cases (the full-size workloads: Sec. 1.1 Eq. stages/update; Sec. 6
Eq. dae_stage for the DAE):

* burgers2d_512_gauss2 / _gauss3: 2D viscous Burgers 512^2, nu = 5e-3,
  dt = 2e-3, random-Fourier initial field (seed 1), 50 steps;
* vsf_1024_gauss5: double shear layer 1024^2, Re = 1000, dt = 5e-3 (seed 2),
  Gauss s = 5, 20 steps.

Run single-threaded (OMP_NUM_THREADS=1); one case takes tens of minutes.
"""
from __future__ import annotations

import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import irk as orc  # noqa: E402
from oracle import vsf as ovsf  # noqa: E402
from oracle.operators import Problem  # noqa: E402

CASES = {
    "burgers2d_512_gauss2": dict(op="burgers2d", n=512, nu=5e-3, dt=2e-3, stages=2, seed=1,
                                 nsteps=50),
    "burgers2d_512_gauss3": dict(op="burgers2d", n=512, nu=5e-3, dt=2e-3, stages=3, seed=1,
                                 nsteps=50),
    "vsf_1024_gauss5": dict(op="vsf", n=1024, nu=1e-3, dt=5e-3, stages=5, seed=2, nsteps=20),
}


def path(case: str) -> str:
    return os.path.join(HERE, f"traj_{case}.npz")


def run(case: str) -> None:
    c = CASES[case]
    n, s, dt = c["n"], c["stages"], c["dt"]
    if c["op"] == "vsf":
        p = Problem("vsf", n, c["nu"], 2 * math.pi)
        u = ovsf.initial_state(workloads.double_shear_layer_vorticity(n, seed=c["seed"]), p.h)
    else:
        p = Problem("burgers2d", n, c["nu"], 1.0)
        u = workloads.random_fourier_2d(n, seed=c["seed"])
    norms = [float(np.linalg.norm(u))]
    its = []
    u1 = None
    t = 0.0
    for k in range(c["nsteps"]):
        t0 = time.perf_counter()
        if c["op"] == "vsf":
            u, _, info = ovsf.reduced_step(p, s, u, t, dt)
        else:
            u, _, info = orc.step(p, s, u, t, dt, linear="gmres")
        t += dt
        norms.append(float(np.linalg.norm(u)))
        its.append(info.iterations)
        if k == 0:
            u1 = u.copy()
        print(f"{case}: step {k + 1}/{c['nsteps']} newton {info.iterations} "
              f"gmres {info.linear_iterations} {time.perf_counter() - t0:.1f} s", flush=True)
        save(case, c, k + 1, norms, its, u, u1)
    print(f"wrote {path(case)}", flush=True)


def save(case: str, c: dict, done: int, norms, its, u, u1) -> None:
    """Write the trajectory so far (after every step, so that an interrupted
    run leaves a valid shorter trajectory: `nsteps` is the steps done)."""
    out = dict(norms=np.array(norms), newton_its=np.array(its),
               **{k: np.array(v) for k, v in c.items() if k not in ("op", "nsteps")})
    out["nsteps"] = np.array(done)
    if c["op"] == "vsf":
        out["u_final"] = u[0]
        out["u_step1"] = u1[0]
    else:
        out["u_final"] = u
    tmp = path(case) + ".tmp.npz"
    np.savez(tmp, **out)
    os.replace(tmp, path(case))


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        run(name)
