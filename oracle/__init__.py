"""FP64 CPU oracle for the Gauss-IRK nonlinear stage solve (test infrastructure).

This package is test infrastructure: only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it.  It shares no code with the
CUDA path and never calls it.

It computes, the plain way, the result the fast method converges to:
u_{n+1} = u_n + dt * sum_i b_i k_i (Eq. update), where k solves the stage
equations M k_i = N(u_n + dt sum_j a_ij k_j, t_n + c_i dt) (Eq. stages) to
a Newton relative residual far below 1e-10, using exact Newton on the fully
coupled sN x sN system (Eq. k0) with a sparse direct solve (or, for grids
where a direct factorisation does not fit, restarted GMRES on the same exact
Jacobian to rtol 1e-13).  For the vorticity-streamfunction DAE (Sec. 6,
Eq. dae_stage) the constraint rows are included in the same Newton system.

Modules
  tableau    Gauss tableau from Legendre nodes; real Schur form of A0^{-1};
             eta/beta/phi/gamma* and the d_{k,l} vectors (Sec. 3.1-3.2, Eq. gamma*)
  operators  Periodic finite-difference N(u,t) and its Jacobian (sparse)
  irk        Stage residual, exact Newton, step driver
  vsf        Vorticity-streamfunction DAE helpers (FFT-eliminated variant)
"""

