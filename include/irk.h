/*
 * irk.h -- C ABI of the GB300 Gauss-IRK nonlinear stage solver.
 *
 * Problem (Sec. 1.1, Eq. problem):  M u'(t) = N(u, t),  u(0) = u0,
 * advanced by an s-stage Gauss Runge-Kutta method (Eq. update, Eq. stages):
 *     u_{n+1} = u_n + dt * sum_i b_i k_i,
 *     0 = M k_i - N(u_n + dt * sum_j a_ij k_j, t_n + c_i dt),   i = 1..s.
 * For the vorticity-streamfunction DAE (Sec. 6, Eq. dae / dae_stage) the state
 * is (omega, psi), M = diag(I, 0) and the second row of N is the constraint
 * G(omega, psi) = -L psi - omega; psi_{n+1} = psi_n + dt sum_i b_i l_i.
 *
 * Each step solves the stage equations by the Newton-like iteration of
 * Algorithm 1 (Sec. 5): the stage block is transformed by the real Schur
 * vectors of A0^{-1} (Sec. 3.1), the 1x1 and 2x2 diagonal blocks D_i of
 * Eq. diag_blocks are solved by flexible GMRES preconditioned by the block
 * lower-triangular L_P of Eq. Lprec with gamma* (Eq. gamma*), and the inner
 * inverses (gamma M - dt L)^{-1} are one geometric-multigrid V-cycle each.
 * N and its Jacobian are built-in periodic finite-difference stencils chosen
 * by `op`; they are not callbacks (device kernels cannot call host code).
 *
 * Conventions
 *  - All floating-point data are IEEE binary64.
 *  - A state vector holds ncomp * n^dim values, component-major; a 2D field is
 *    row-major [y][x] (x fastest).  ncomp = 1 for the 1D operators, 2 for
 *    Burgers-2D (u, v) and VSF (omega, psi).  A stage block holds s states,
 *    stage-major.
 *  - `*_on_device` = 1 means the pointer is CUDA device memory on the current
 *    device (e.g. a torch tensor's data_ptr()); 0 means host memory.
 *  - A handle lives on the device that was current at irk_create.  Every call
 *    on it makes that device current while it runs and gives the caller's
 *    current device back on return.
 *  - The caller owns every buffer it passes; the library copies in and out.
 *    The handle owns all device memory it allocates (one arena, sized at
 *    irk_create) and releases it in irk_destroy.
 *  - Work is issued on the stream given to irk_create (NULL = a stream the
 *    library creates).  Calls return after their results are complete.
 *  - Every call returns a status.  A failed irk_step leaves the state at the
 *    last accepted step.  irk_last_error() describes the most recent failure.
 *  - Calls on one handle must not overlap; distinct handles are independent.
 */
#ifndef IRK_H
#define IRK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct irk_handle irk_handle;

typedef enum {
  IRK_OK = 0,
  IRK_ERR_INVALID = 1,          /* bad argument or unsupported configuration */
  IRK_ERR_NOMEM = 2,            /* device or host allocation failed */
  IRK_ERR_CUDA = 3,             /* a CUDA runtime call failed */
  IRK_ERR_NEWTON_DIVERGED = 4,  /* non-finite or growing stage residual */
  IRK_ERR_NEWTON_MAXIT = 5,     /* residual tolerance not met in newton_maxit */
  IRK_ERR_KRYLOV_BREAKDOWN = 6, /* FGMRES lost its basis or did not converge */
  IRK_ERR_TIMEOUT = 7,          /* a bounded device wait gave up */
  IRK_ERR_NO_DEVICE = 8         /* no CUDA device is available */
} irk_status;

/* Runge-Kutta families with A0 invertible and A0^{-1} positive stable (the
 * standing assumption of Sec. 2; Table 1 covers the first three).  SDIRK is
 * the diagonally implicit comparison of Sec. 7 (Tables ev-solvers,
 * naca-iters, dsl-iters; DIRK background in Sec. 2.1): lower
 * triangular A0 with one diagonal value gamma, stiffly accurate, L-stable. */
typedef enum {
  IRK_GAUSS = 0,        /* order 2s */
  IRK_RADAU_IIA = 1,    /* order 2s-1, stiffly accurate */
  IRK_LOBATTO_IIIC = 2, /* order 2s-2, s >= 2 */
  IRK_SDIRK = 3         /* s = 1, 2, 3, 5: order 1, 2, 3, 4 (backward Euler;
                           gamma = 1 - sqrt(1/2); Alexander's 3-stage method;
                           the 5-stage order-4 method of Hairer and Wanner) */
} irk_family;

/* Basis of the A0^{-1} transform in Algorithm 1 (Sec. 3.1). */
typedef enum {
  IRK_BASIS_SCHUR = 0,  /* standardized real Schur form Q0 R0 Q0^T (default) */
  IRK_BASIS_EIGEN = 1   /* real eigenvector basis T R T^{-1}, R block diagonal */
} irk_basis;

typedef enum {
  IRK_OP_DIFFUSION_1D = 0, /* N = nu D2 u                       (linear test)   */
  IRK_OP_BURGERS_1D = 1,   /* N = -(u_{i+1}^2 - u_{i-1}^2)/(4h) + nu D2 u        */
  IRK_OP_BURGERS_2D = 2,   /* N = (-u Dx u - v Dy u + nu L u, same for v)        */
  IRK_OP_VSF_2D = 3        /* N = (J_A(psi, omega) + nu L omega, -L psi - omega) */
} irk_op;

typedef enum { IRK_MASS_IDENTITY = 0, IRK_MASS_DAE = 1 } irk_mass;

/* Storage and arithmetic of the V-cycle preconditioner (Newton residual,
 * stage updates, FGMRES and its Gram-Schmidt stay FP64 in every case):
 * FP64 everything FP64; FP32 vectors and operator data in FP32 with FP32
 * arithmetic; BF16 the operator data (the velocity of every level) stored in
 * BF16, vectors (iterates, right-hand sides, residuals) in FP32, FP32
 * arithmetic. */
typedef enum { IRK_MG_FP64 = 0, IRK_MG_FP32 = 1, IRK_MG_BF16 = 2 } irk_mg_precision;

typedef struct {
  int family;        /* irk_family */
  int stages;        /* s, 1..5 */
  int op;            /* irk_op */
  int mass;          /* irk_mass; must be IRK_MASS_DAE exactly for IRK_OP_VSF_2D */
  int n;             /* grid points per dimension, power of two, 8..8192 */
  double length;     /* periodic domain [0, length)^dim */
  double nu;         /* viscosity (1/Re for VSF), > 0 */
  int forcing;       /* 0, or 1 = manufactured source of the 1D operators */
  double newton_rtol;   /* stop at ||F(k)|| <= newton_rtol ||F(0)||; default 1e-10 */
  int newton_maxit;     /* default 20 */
  double krylov_rtol;   /* loosest FGMRES relative tolerance per block; default 1e-3 */
  int krylov_restart;   /* FGMRES(m) restart length m, 1..64; default 30 */
  int krylov_maxit;     /* total FGMRES iterations per block solve; default 200 */
  int nonlinear_variant;/* nonlinear iteration (Sec. 3.2); default 2:
                           0 simplified Newton: every diagonal block uses the
                             Jacobian at the last stage state;
                           1 block diagonal, each block lumped onto the stage
                             of its largest d-vector entry;
                           2 block diagonal (d_ii^T L-hat); the same as 3 for
                             2-stage Gauss (Q0 = I) and SDIRK (no coupling);
                           3 block upper triangular within the pattern of R0
                             (exact Newton for s = 2);
                           4 exact Newton: an outer FGMRES on the true stage
                             Jacobian, right-preconditioned by one
                             Algorithm-1 sweep of variant 3 */
  int gamma_mode;       /* 0: gamma* = eta + beta^2/eta (Eq. gamma*), 1: gamma = eta */
  int mg_precision;     /* irk_mg_precision of the V-cycle preconditioner */
  int mg_levels;        /* 0 = coarsen down to the coarsest size below */
  int mg_pre, mg_post;  /* damped-Jacobi sweeps per level (rows that are not
                           shift-dominated, see mg_shifted_sweeps); default 2, 2 */
  int mg_coarse_sweeps; /* sweeps on the coarsest level; default 40 */
  double mg_omega;      /* Jacobi damping; 0 = default (0.8 in 2D, 2/3 in 1D) */
  int profile;          /* 1 = time each kernel class with CUDA events */
  int use_graphs;       /* 1 (default) = run each IRK step as one CUDA graph
                           (Newton and FGMRES loops in conditional nodes),
                           captured once per dt; forced off while profile = 1 */
  int initial_guess;    /* Newton start (the tolerance is relative to
                           ||F(k=0)|| in every case):
                           2 (default) = the previous step's stages
                             extrapolated along the collocation polynomial
                             (Gauss, Radau IIA: k_j = sum_i k_i l_i(1 + c_j
                             dt/dt_prev), l_i the Lagrange basis on the
                             abscissae); other families use them as they are;
                           1 = the previous step's stages;
                           0 = zero.
                           irk_set_state resets the stages to zero;
                           irk_set_stages marks the given stages as from a
                           step of the next step's dt */
  int basis;            /* irk_basis; default IRK_BASIS_SCHUR */
  int mg_shifted_sweeps;/* pre- and post-sweeps on shift-dominated rows of 2D
                           grids (sigma >= 0.15 D on the finest level, D the
                           Jacobi diagonal), where more smoothing does not
                           lower the Krylov counts; default 1; 0 = mg_pre/mg_post */
  double mg_coarse_reduction; /* error reduction the Jacobi sweeps target on a
                           shift-dominated coarsest level (2..12 sweeps);
                           default 2e-2; 0 = default */
  int mg_coarse_smoother; /* sweeps on a shift-dominated 2D coarsest level
                           (n >= 32) toward mg_coarse_reduction:
                           0 (default) undamped Jacobi, in fused pairs;
                           1 Chebyshev-accelerated Jacobi;
                           2 red-black Gauss-Seidel, one sweep per launch,
                             half the sweeps of Jacobi */
  int dirk_sequential;  /* IRK_SDIRK only: 1 (default) = solve the stages one
                           after another, each a nonlinear solve of
                           M k_i = N(u_n + dt sum_{j<i} a_ij k_j + dt gamma k_i)
                           with its own Newton loop (the usual DIRK solve);
                           0 = Algorithm 1 over the coupled stage system (the
                           transformed Jacobian is exactly block upper
                           triangular, so variant 3 is exact Newton there) */
  int dae_solver;       /* IRK_OP_VSF_2D only (Sec. 7.2): 0 (default) = FGMRES
                           on each (omega, psi) block of Eq. vsf-system-1 with
                           one omega V-cycle and one psi V-cycle per
                           preconditioner application; 1 = block forward
                           solve of the reordered Picard system Eq.
                           vsf-system-2: FGMRES on the omega block to
                           krylov_rtol, then one MG-preconditioned FGMRES
                           Poisson solve per stream function row */
  int mg_tile_rows;     /* rows of the 32-wide tiles of the three-sweep V-cycle
                           kernel: 0 (default) = 16 with FP64 storage, 8
                           otherwise; 8 or 16 to fix it (an autotuner knob) */
  int mg_fuse_transfer; /* 2D levels of n >= 32 whose single pre-sweep is
                           folded into the residual: 1 = one kernel forms
                           the residual and restricts it; 2 = two kernels
                           and a stored residual; 0 (default) = 1 with
                           FP32/BF16 storage, 2 with FP64 (measured faster
                           there: the fused kernel's FP64 stencil work is
                           not hidden).  Same result bit for bit; an
                           autotuner knob */
} irk_config;

typedef struct {
  int steps;            /* accepted steps in this call */
  int newton_its;       /* Newton iterations (summed over steps) */
  int krylov_its;       /* FGMRES iterations (summed over blocks and steps) */
  int prec_apps;        /* preconditioner applications: 1 per 1x1 and 2 per 2x2
                           Krylov iteration (counting rule of Sec. 7.1.1) */
  int vcycles;          /* V-cycles applied */
  int max_newton_its;   /* worst step */
  double final_rel_res; /* ||F|| / ||F(0)|| at acceptance of the last step */
  long long kernel_launches; /* this library's kernel launches in the call */
  int outer_its;        /* variant 4: outer FGMRES iterations on the true Jacobian */
  int poisson_vcycles;  /* VSF: V-cycles on the stream function Poisson block
                           (included in vcycles) */
} irk_stats;

typedef struct {
  char name[32];        /* kernel class */
  long long launches;
  double ms;            /* summed CUDA-event time of its launches */
  double bytes;         /* summed algorithmic DRAM bytes (minimum traffic) */
  double flops;         /* summed algorithmic floating-point operations */
} irk_kernel_stat;

/* Fill *cfg with the defaults listed above (Gauss s=2, Burgers-1D n=256). */
void irk_config_default(irk_config* cfg);

/* Create a solver for cfg with initial state u0 (ncomp*n^dim values).
 * For IRK_OP_VSF_2D only omega is read from u0 (first n^2 values); psi is
 * made consistent by solving -L psi = omega (zero mean) on the device.
 * cuda_stream: a cudaStream_t, or NULL.  Validation (Assumption 1, Sec. 2.2):
 * rejects s outside 1..5, n not a power of two, nu <= 0, a mass that does not
 * match op.  On success *out owns the device arena. */
irk_status irk_create(const irk_config* cfg, const double* u0, int u0_on_device,
                      void* cuda_stream, irk_handle** out);

/* Device bytes the arena of a handle for cfg needs (host-only, no GPU);
 * 0 if cfg is invalid. */
size_t irk_config_device_bytes(const irk_config* cfg);

/* As irk_create, but the handle carves its arena out of caller-owned device
 * memory (256-byte aligned, at least irk_config_device_bytes(cfg) bytes) and
 * never frees it.  Used by memory managers that own the device pool (the
 * serving runtime below). */
irk_status irk_create_in(const irk_config* cfg, const double* u0, int u0_on_device,
                         void* cuda_stream, void* arena, size_t arena_bytes, irk_handle** out);

/* Advance nsteps steps of size dt from time t_n (Algorithm 1 per step).
 * stats may be NULL. */
irk_status irk_step(irk_handle* h, double t_n, double dt, int nsteps, irk_stats* stats);

/* Copy the current state out / in (ncomp*n^dim values; VSF: omega then psi). */
irk_status irk_get_state(irk_handle* h, double* dst, int dst_on_device);
irk_status irk_set_state(irk_handle* h, const double* src, int src_on_device);

/* irk_set_state for a caller that streams one trajectory through host
 * memory: replaces the state but keeps the stages of the last accepted step
 * as the basis of the next Newton guess (initial_guess 1 or 2).  The tolerance stays relative
 * to ||F(k=0)||, so the fixed point does not depend on the guess; for an
 * unrelated state use irk_set_state, which starts from zero stages. */
irk_status irk_set_state_keep_stages(irk_handle* h, const double* src, int src_on_device);

/* Stage vectors k_1..k_s of the last accepted step (s*ncomp*n^dim values). */
irk_status irk_get_stages(irk_handle* h, double* dst, int dst_on_device);

/* Set the stage vectors the next step's Newton starting guess is formed from
 * (initial_guess 1 or 2; for 2 they count as stages of a step of the next
 * step's dt).  A checkpoint that must resume bit for bit saves the state and
 * the stages and restores both, the stages after the state. */
irk_status irk_set_stages(irk_handle* h, const double* src, int src_on_device);

/* Stage residual F_i = M k_i - N(u + dt sum_j a_ij k_j, t_n + c_i dt)
 * (Eq. stages) of a caller-given stage block K about the current state.
 * K and F hold s*ncomp*n^dim values. */
irk_status irk_stage_residual(irk_handle* h, double t_n, double dt, const double* K,
                              double* F, int on_device);

/* Jacobian-vector product of the stage equations (Eq. k0):
 * (J V)_i = M v_i - dt N'(Y_i) sum_j a_ij v_j with Y_i the stage states of K. */
irk_status irk_stage_jacobian_apply(irk_handle* h, double dt, const double* K,
                                    const double* V, double* JV, int on_device);

/* Stage residual without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- a host
 * whose memory manager owns the device pool and forbids raw allocations, a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the device,
 * or an embedding with a fixed device-memory budget.
 *
 * Computes F_i = M k_i - N(u + dt sum_j a_ij k_j) for the autonomous operator
 * `op` (no forcing) on a periodic n^dim grid of spacing length/n, and
 * *fnorm = ||F||_2.  A is the s x s Butcher matrix (host, row-major; e.g. from
 * irk_tableau).  u (ncomp*n^dim), K and F (s*ncomp*n^dim) and fnorm (one
 * double) are caller-owned DEVICE pointers; the work is enqueued on
 * cuda_stream (NULL = the legacy default stream) and the call returns without
 * waiting for it.
 *
 * Scratch: a fixed 32 KiB file-scope device array (one partial sum per 256
 * grid points) that every GPU loading the library keeps until exit.  Limit:
 * n^dim <= 1,048,576 points (e.g. 1024^2); larger grids return IRK_ERR_NOMEM
 * with a message on stderr and launch nothing.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and caches it;
 * make that first call before any stream capture.  The cache lives as long
 * as the process: after cudaDeviceReset on that device the cached address is
 * stale, so do not call this entry again in such a process.  Every call
 * shares the array and leaves its partials there (each call rewrites every
 * slot it reads, so nothing needs clearing); calls whose work overlaps on
 * the GPU, e.g. on two streams, race on it.  u, K, F and fnorm must be
 * device (or managed) memory of the current device, checked with
 * cudaPointerGetAttributes before anything is launched; a buffer on another
 * device or in host memory, and any other bad argument, returns
 * IRK_ERR_INVALID. */
irk_status irk_stage_residual_noalloc(int op, int n, double length, double nu, int stages,
                                      const double* A, double dt, const double* u,
                                      const double* K, double* F, double* fnorm,
                                      void* cuda_stream);

/* Host-only: tableau of `family` with s stages and the standardized real Schur
 * form A0^{-1} = Q0 R0 Q0^T (Sec. 3.1).  A, Q0, R0 are s*s row-major; b, c
 * length s; block_sizes receives the diagonal block sizes (1 or 2) in order,
 * *nblocks their count.  Needs no GPU. */
irk_status irk_tableau(int family, int s, double* A, double* b, double* c,
                       double* Q0, double* R0, int* block_sizes, int* nblocks);

/* Host-only: the A0^{-1} transform of Algorithm 1 in either basis,
 * A0^{-1} = T R T^{-1} (Sec. 3.1).  T, Tinv, R are s*s row-major (T = Q0,
 * Tinv = Q0^T, R = R0 for IRK_BASIS_SCHUR); block_sizes and *nblocks as for
 * irk_tableau.  Any output pointer may be NULL.  Unknown family or basis, or
 * s out of range, returns IRK_ERR_INVALID.  Needs no GPU. */
irk_status irk_transform(int family, int s, int basis, double* T, double* Tinv, double* R,
                         int* block_sizes, int* nblocks);

/* The handle's current settings (after irk_autotune, the chosen ones). */
irk_status irk_get_config(const irk_handle* h, irk_config* out);

/* Empirical tuning of the V-cycle preconditioner on the handle's own
 * workload.  From the current state and stages, each candidate setting is
 * timed over `steps` IRK steps of size dt (after one untimed step that
 * captures its graphs), by CUDA events on the handle's stream; candidates
 * come by coordinate descent over mg_shifted_sweeps {1, 2},
 * mg_coarse_smoother {0, 2}, mg_coarse_reduction {2e-2, 5e-3}, mg_tile_rows
 * {8, 16}, mg_levels {0 (automatic), automatic depth + 1} and
 * mg_fuse_transfer {1, 2}, starting from the current settings, and the
 * fastest is kept.  A candidate whose
 * step fails is skipped.  State and stages are restored afterwards, and the
 * statistics of the trial steps are discarded.  Allocates a backup of the
 * state and stages (cudaMalloc) for the duration of the call.  The choice
 * depends on measured times and can differ between runs; every candidate
 * reaches the same Newton tolerance.  *chosen (may be NULL) receives the
 * kept settings.  1 <= steps <= 100. */
irk_status irk_autotune(irk_handle* h, double t_n, double dt, int steps, irk_config* chosen);

/* Per-kernel-class timing gathered while cfg.profile = 1 (CUDA events on the
 * handle's stream).  Writes up to max entries, *count = entries written. */
irk_status irk_kernel_stats(irk_handle* h, irk_kernel_stat* out, int max, int* count);
irk_status irk_reset_kernel_stats(irk_handle* h);

/* Measurement utility; the paper has no counterpart.  Measures the fused
 * multiply-add throughput of the current device in TFLOP/s (one FMA = two
 * operations), the roofline ceiling of kernels bound by floating-point
 * arithmetic: precision 0 = FP64, 1 = FP32.  Runs independent FMA chains on
 * 8 blocks of 256 threads per SM on cuda_stream (NULL = legacy default
 * stream), timed by CUDA events, best of five runs of about 20 ms after one
 * calibration run; allocates and frees one small output buffer.  Blocks until
 * done.  Other precision values or a NULL tflops return IRK_ERR_INVALID. */
irk_status irk_measure_alu_peak(int precision, void* cuda_stream, double* tflops);

/* Device bytes held by the handle's arena. */
size_t irk_device_bytes(const irk_handle* h);

/* Human-readable text of the last failure on h (valid until the next call on
 * h), or, when h is NULL, of the calling thread's last failed irk_create. */
const char* irk_last_error(const irk_handle* h);
const char* irk_status_string(irk_status st);

/* Release the handle and its device memory.  NULL-safe. */
void irk_destroy(irk_handle* h);

/* Bounds-checked debug build only (the library compiled with -DIRK_BOUNDS).
 * There, the device index checks of the kernels (grid neighbours, multigrid
 * tiles and transfers, Krylov basis columns) do not access memory out of
 * range.  Each out-of-range index counts a hit in a per-source-file device
 * record and is replaced by 0.  irk_step collects the records after every
 * step and fails the step (IRK_ERR_CUDA, the first hit in irk_last_error) if
 * any hit was recorded.  This call returns the hits recorded since the last
 * collection and clears them.  It writes the first hit's file, line, index and
 * extent to msg (msg_len bytes including the terminator; msg may be NULL).
 * selftest != 0 first runs a one-thread kernel that checks index 1 against
 * extent 1; the check records one hit and redirects the store to index 0.
 * Returns -1 in the normal build (needs no GPU there), -2 if a CUDA call
 * fails.  Not thread-safe: the records are global to the process. */
long long irk_debug_bounds(int selftest, char* msg, size_t msg_len);

#ifdef __cplusplus
}
#endif

#endif /* IRK_H */
