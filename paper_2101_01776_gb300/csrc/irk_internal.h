// Internal declarations shared by the solver's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/irk.h"
#include "bounds.h"

#define IRK_MAXS 5
#define IRK_MAX_TERMS 5
#define IRK_MAX_COMBOS (IRK_MAXS * IRK_MAXS)
#define IRK_MAX_LEVELS 16
#define IRK_BLAS_THREADS 256
#define IRK_FG_MAXM 64

namespace irk {

// Programmatic dependent launch.  The solver's kernels are launched with
// launch_pdl: a kernel may be scheduled while its predecessor on the stream
// (or in the captured graph) is still draining, so its launch latency hides
// behind that kernel's tail.  Every such kernel begins with pdl_entry(): it
// waits until the predecessor grid has completed and its writes are visible
// (so no global access of the kernel can race with it) and then lets its own
// successor be scheduled.  For a kernel launched without the attribute both
// instructions return at once.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
#endif

// Makes `dev` (a handle's device) current for the scope of an API call and
// gives the caller's current device back on return, so that a call made while
// another device is current allocates, copies and launches on the handle's
// device and not on that one.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
      return;
    }
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
};

// The error of the launch is left for the caller's cudaGetLastError, as with
// the <<<>>> syntax.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#ifdef IRK_BOUNDS
// per-translation-unit records of the bounds-checked build (bounds.h)
int bounds_take_stencil(BoundsRecord* out);
int bounds_take_mg(BoundsRecord* out);
int bounds_take_blas(BoundsRecord* out);
int bounds_take_fgmres(BoundsRecord* out);
int bounds_take_noalloc(BoundsRecord* out);
// one thread checks index 1 against extent 1 (one hit in blas.cu's record)
// and stores through the checked index, which the check turns into 0
void launch_bounds_selftest(cudaStream_t st);
// Hits of every translation unit's record since the last collection (the
// records are cleared), the first hit described in *msg; -1 when a CUDA call
// fails.
long long bounds_collect(std::string* msg);
#endif

// Host-side trace ranges in the NVTX domain "irk": API calls, steps, Newton
// iterations, block solves, V-cycles.  With no tool attached (no
// NVTX_INJECTION64_PATH) a push/pop is one indirect call to a no-op.  Inside a
// captured CUDA graph the ranges mark the capture, not the replay.
inline nvtxDomainHandle_t trace_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("irk");
  return d;
}
struct TraceRange {
  explicit TraceRange(const char* name) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(trace_domain(), &a);
  }
  ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// A0^{-1} = T R T^{-1}: T = Q0 (orthogonal, T^{-1} = Q0^T) and R = R0 in the
// real Schur basis; T = real eigenvectors and R block diagonal otherwise.
struct HostTableau {
  int s;
  double A[IRK_MAXS * IRK_MAXS], b[IRK_MAXS], c[IRK_MAXS];
  double Ainv[IRK_MAXS * IRK_MAXS], T[IRK_MAXS * IRK_MAXS], Tinv[IRK_MAXS * IRK_MAXS];
  double R[IRK_MAXS * IRK_MAXS];
  double TR[IRK_MAXS * IRK_MAXS];  // T R: back-transform of Algorithm 1
  int nblk, bstart[IRK_MAXS], bsize[IRK_MAXS];
  double eta[IRK_MAXS], beta2[IRK_MAXS], gamma_star[IRK_MAXS];
  int collocation;  // Gauss, Radau IIA: k_i = u'(t_n + c_i dt) of the collocation polynomial
};

int build_tableau(int family, int s, int basis, HostTableau* t, char* err, size_t errlen);
// Internal Newton status of the device loop: the warm-start guess has a
// larger residual than zero stages; the step restarts from zero.
constexpr int kGuessRejected = 100;
// a warm start counts as worse than zero stages above this ||F(guess)|| / ||F(0)||
// (margin over 1: the two norms are summed in different orders)
constexpr double kGuessLimit = 1.001;
// The single-stage tableau A = [gamma], b = [1], c = [0] (one SDIRK stage
// solved on its own); nonzero for gamma <= 0.
int build_tableau_single(double gamma, HostTableau* t);

// ---------------------------------------------------------------------------
// Grid and operator description passed to every stencil kernel.
struct GridDesc {
  int dim;       // 1 or 2
  int n;         // points per dimension (power of two)
  int logn;
  int npts;      // n^dim
  int ncomp;     // state components
  int op;        // irk_op
  double h, inv2h, inv4h, invh2, inv12h2;
  double nu;
};

// Pointwise stage states and combined fields (steps a2 + a7 setup):
//   Y_i = u + dt sum_j A_ij K_j ;  Ybar_q = sum_m D_qm Y_m
struct StageStateArgs {
  int s, ncombo;
  long long L;           // ncomp * npts
  double dt;
  double A[IRK_MAXS * IRK_MAXS];
  double D[IRK_MAX_COMBOS * IRK_MAXS];  // ncombo x s
  const double* u;       // may be null (treated as 0)
  const double* K;       // s * L
  double* Y;             // s * L (may be null)
  double* combos;        // ncombo * L (may be null)
};

// Stage residual (step a3) with the Algorithm-1 RHS transform (step a5):
//   F_i = M K_i - N(Y_i, t_n + c_i dt);  rhs_k = -sum_i Q0_{ik} F_i ; partial ||F||^2
struct ResidualArgs {
  int s;
  double Q[IRK_MAXS * IRK_MAXS];
  double tstage[IRK_MAXS];
  int forcing;
  const double* Y;       // s * L
  const double* K;       // s * L
  double* rhs;           // s * L, may be null
  double* Fraw;          // s * L, may be null (untransformed residual)
  double* partials;      // one per block
};

// Generic block operator (steps a6, a7, a9 coupling):
//   y_r = alpha * base_r + sigma * sum_t [ m_t M x_t - dt ( Jadv(Ybar_t) x_t + lin_t Jlin x_t ) ]
struct OpTerm {
  const double* x;       // ncomp * npts
  const double* combo;   // ncomp * npts or null (no advective part)
  const double* coef;    // coefficient fields of `combo` at this dt (launch_combo_coef:
                         // 6 * npts Burgers-2D, 16 * npts VSF), or null: formed per point
  double m;              // mass coefficient
  double lin;            // coefficient of the state-independent linear part
  double kd, cc;         // set by launch_stage_op: dt lin nu / h^2 and m + 4 kd
};
struct OpRow {
  double* y;
  const double* base;    // may be null
  double alpha, sigma;
  int nterm;
  OpTerm t[IRK_MAX_TERMS];
};
struct StageOpArgs {
  int nrow;
  double dt;
  OpRow row[2];
  double* copy_dst;      // optional: copy_src -> copy_dst (ncomp*npts*copy_rows)
  const double* copy_src;
  long long copy_len;
  const int* copy_jdev;  // optional: copy_dst += (*copy_jdev) * copy_ldv (device index)
  long long copy_ldv;
  int vsf_omega_only;    // VSF: rows and terms hold omega alone (Picard omega block)
};

// Device-resident FGMRES(m) state of one block solve (Arnoldi/Givens data).
struct FGState {
  int j;          // current Arnoldi index
  int k;          // columns of the final least-squares problem
  int its;        // iterations of this cycle
  int status;     // 0 ok, 2 non-finite
  int stopped;    // the loop has ended (set by the Arnoldi step)
  int guard;      // body executions this cycle (independent loop bound)
  unsigned int ctr1, ctr2;  // last-block counters of the fused CGS2 kernels
  double beta, target, res, inv_scale;
  double g[IRK_FG_MAXM + 1];
  double cs[IRK_FG_MAXM], sn[IRK_FG_MAXM], y[IRK_FG_MAXM];
  double H[IRK_FG_MAXM * (IRK_FG_MAXM + 1)];  // column-major, column j at j*(MAXM+1)
};

// ---------------------------------------------------------------------------
// Multigrid level (one scalar-operator hierarchy, all state components).
struct MGLevelDesc {
  int n, logn, npts;
  double h;
};

// MG_ADVECTIVE_PRE: MG_ADVECTIVE on a 2D grid with the four off-diagonal
// coefficients precomputed per point (launch_mg_coef): the `vel` argument of
// the MG kernels then holds 4 fields (E, W, N, S) instead of the velocity.
enum MGKind { MG_ADVECTIVE = 0, MG_CONSERVATIVE_1D = 1, MG_DIFFUSION = 2, MG_ADVECTIVE_PRE = 3 };

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files).
void launch_stage_states(const GridDesc& g, const StageStateArgs& a, cudaStream_t st);
int residual_blocks(const GridDesc& g);
void launch_residual(const GridDesc& g, const ResidualArgs& a, cudaStream_t st);
void launch_stage_op(const GridDesc& g, const StageOpArgs& a, cudaStream_t st);
void launch_neg_laplacian(const GridDesc& g, const double* x, double* y, cudaStream_t st);
// Burgers-2D coefficient fields of each combined field (ub, vb), formed once
// per Newton iteration: dt ub/(2h), dt vb/(2h), dt Dx ub, dt Dy ub, dt Dx vb,
// dt Dy vb (central differences); coef is ncombo * 6 * npts
// Combined fields that get coefficient fields: slot i of coef belongs to
// combined field idx[i] (the fields of the diagonal blocks, read every Krylov
// iteration; the upper-coupling fields are read once per Newton iteration)
struct ComboList {
  int n;
  int idx[IRK_MAX_COMBOS];
};
void launch_combo_coef(const GridDesc& g, const double* combos, const ComboList& list, double dt,
                       double* coef, cudaStream_t st);
// coefficient fields per combined field for `op` (6 Burgers-2D, 16 VSF: the
// dt/(12h^2)-scaled Arakawa weights of psibar and wbar), 0 = none
int combo_coef_fields(int op);
// K_j <- sum_i E_ji K_i per point, E (s x s, row-major) read from device memory
void launch_stage_extrapolate(long long L, int s, const double* E, double* K, cudaStream_t st);
void launch_stage_update(long long L, int s, const double* QR, const double* yhat, double* K,
                         cudaStream_t st);
void launch_u_update(long long L, int s, const double* b, double dt, const double* K, double* u,
                     cudaStream_t st);
void launch_velocity_from_combo(const GridDesc& g, const double* combo, void* vel, int prec,
                                cudaStream_t st);
void launch_remove_mean(long long npts, int nfields, long long stride, double* x, double* scratch,
                        cudaStream_t st);

// BLAS-1 for FGMRES (FP64, deterministic reductions)
int blas_blocks(long long L);
void launch_multi_dot(const double* V, long long ldv, int nv, const double* w, long long L,
                      double* partials, cudaStream_t st);
void launch_update_dot(const double* V, long long ldv, int nv, const double* hdev, double* w,
                       long long L, int with_dots, double* partials, cudaStream_t st);
void launch_reduce(const double* partials, int nblk, int stride, int nvals, double* out,
                   cudaStream_t st);
void launch_scale_copy(const double* w, double scale, double* v, double* v2, long long L,
                       cudaStream_t st);
void launch_lincomb(double* x, const double* Z, long long ldz, int k, const double* y,
                    long long L, cudaStream_t st);
void launch_norm2(const double* x, long long L, double* partials, cudaStream_t st);
void launch_axpby(double* y, double a, const double* x, double b, long long L, cudaStream_t st);

// Device-resident FGMRES (fgmres_dev.cu)
void launch_fg_init(FGState* s, const double* nrm2, const double* rtol,
                    cudaGraphConditionalHandle cond, cudaStream_t st);
void launch_fg_scale(const double* w, const FGState* s, double* V, long long ldv, double* prec_in,
                     long long L, cudaStream_t st);
void launch_fg_solve(FGState* s, cudaStream_t st);
void launch_zero_if_unforced(const double* nw, double* K, long long len, cudaStream_t st);
void launch_newton_first(double* nw, const double* f2, double f2_scale, double* rtol_slot,
                         double newton_rtol, double krylov_rtol, cudaGraphConditionalHandle cond,
                         cudaStream_t st);
void launch_newton_ctl(double* nw, const double* f2, double* rtol_slot, double newton_rtol,
                       int maxit, double krylov_rtol, cudaGraphConditionalHandle cond, int count,
                       cudaStream_t st);
// fused CGS2 iteration: dots (+reduce), update+dots (+reduce, Arnoldi step),
// next basis vector (second update fused with the normalisation)
void launch_fg_gs1(const double* V, long long ldv, FGState* s, const double* w, long long L,
                   double* partials, double* h1, cudaStream_t st);
void launch_fg_gs2(const double* V, long long ldv, FGState* s, const double* h1, double* w,
                   long long L, double* partials, double* h2, int m, int maxit, double* its_total,
                   cudaGraphConditionalHandle cond, cudaStream_t st);
void launch_fg_next(const double* V_, long long ldv, FGState* s, const double* h2,
                    const double* w, double* V, double* prec_in, long long L, int guard_limit,
                    cudaGraphConditionalHandle cond, cudaStream_t st);
void launch_fg_lincomb(double* x, const double* Z, long long ldz, const FGState* s, long long L,
                       cudaStream_t st);

// Multigrid (templated on the storage precision; prec = irk_mg_precision)
void launch_mg_smooth(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                      double cadv, double cdiff, double omega, const void* vel, const void* b,
                      const void* w_in, void* w_out, int first, cudaStream_t st,
                      double* epi_out = nullptr, const double* epi_base = nullptr,
                      double epi_coef = 0.0, double epi_bcoef = 1.0,
                      const double* b64 = nullptr, double* out64 = nullptr);
bool mg_smooth2_pays(int prec, int dim, int kind, const MGLevelDesc& lv, int first);
bool mg_smooth3_pays(int prec, int dim, const MGLevelDesc& lv);
// The four off-diagonal coefficients of the 2D advective level operator,
// coef = (beta + alpha a_x, beta - alpha a_x, beta + alpha a_y, beta - alpha a_y)
// with alpha = cadv/(2h), beta = -cdiff/h^2, from the level velocity vel (2 fields)
// Velocity and coefficients of the two finest 2D levels in one launch (FP64)
void launch_mg_setup2(const MGLevelDesc& fine, const MGLevelDesc& coarse, double cadv, double cdiff,
                      const double* combo, void* vel0, void* coef0, void* vel1, void* coef1,
                      cudaStream_t st);
void launch_mg_coef(int prec, const MGLevelDesc& lv, double cadv, double cdiff, const void* vel,
                    void* coef, cudaStream_t st);
// The bottom of a periodic 2D Poisson V-cycle (levels lv.n = 32 or 16 down to
// 8) in one CTA; pinv is the 64 x 64 zero-mean pseudo-inverse of the 8^2
// operator -L_h for cdiff = 1 (device memory, row-major)
void launch_mg_bottom(int prec, const MGLevelDesc& lv, double cdiff, double omega, int pre,
                      int post, const double* pinv, const void* b, void* w, cudaStream_t st);
// Three damped-Jacobi sweeps in one launch (2D, n >= 32), bit-equal to three
// single sweeps: w_in -> w_out (w_in unused when first: w = 0)
void launch_mg_smooth3(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                       double cadv, double cdiff, double omega, const void* vel, const void* b,
                       const void* w_in, void* w_out, int first, cudaStream_t st,
                       int tile_rows = 0);
// One undamped red-black Gauss-Seidel sweep (2D, n >= 32): w_in -> w_out
// (w_in unused when first: w = 0)
void launch_mg_rbgs(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                    double cadv, double cdiff, const void* vel, const void* b, const void* w_in,
                    void* w_out, int first, cudaStream_t st);
// Two Chebyshev-accelerated undamped Jacobi sweeps (2D, n >= 32): from x_prev
// (x_{k-1}) and x_cur (x_k) to x_mid (x_{k+1}) and x_out (x_{k+2}) with the
// three-term weights wa, wb; `first` starts from x_0 = 0
void launch_mg_cheb2(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                     double cadv, double cdiff, const void* vel, const void* b, const void* x_prev,
                     const void* x_cur, void* x_mid, void* x_out, double wa, double wb, int first,
                     cudaStream_t st);
void launch_mg_smooth2(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                       double cadv, double cdiff, double omega, const void* vel, const void* b,
                       const void* w_in, void* w_out, int first, cudaStream_t st);
void launch_mg_residual(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp,
                        double sigma, double cadv, double cdiff, const void* vel, const void* b,
                        const void* w, void* r, cudaStream_t st);
void launch_mg_restrict(int prec, int dim, const MGLevelDesc& fine, int ncomp, const void* rf,
                        void* bc, cudaStream_t st);
// w_f = dinv b_f + P e_c: the prolongation onto a level whose only pre-sweep
// started from zero and was folded into launch_mg_residual0
// b64 / out64 (FP32 and BF16 storage, finest level): b read from the FP64
// input, the result written to the FP64 output (no conversion launches)
void launch_mg_prolong_set(int prec, int dim, const MGLevelDesc& fine, int ncomp, double sigma,
                           double cadv, double cdiff, double omega, const void* bf, const void* wc,
                           void* wf, cudaStream_t st, const double* b64 = nullptr);
// r = b - A (dinv b): the residual after one damped-Jacobi sweep from zero
void launch_mg_residual0(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp,
                         double sigma, double cadv, double cdiff, double omega, const void* vel,
                         const void* b, void* r, cudaStream_t st, const double* b64 = nullptr);
// launch_mg_residual0 and launch_mg_restrict in one launch (2D, fine n >= 32,
// ncomp <= 2): the coarse right-hand side bc, bit for bit, without storing r
void launch_mg_resid0_restrict(int prec, int kind, const MGLevelDesc& fine, int ncomp,
                               double sigma, double cadv, double cdiff, double omega,
                               const void* vel, const void* b, void* bc, cudaStream_t st,
                               const double* b64 = nullptr);
void launch_mg_prolong_add(int prec, int dim, const MGLevelDesc& fine, int ncomp, const void* wc,
                           void* wf, cudaStream_t st);
void launch_mg_coarse(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                      double cadv, double cdiff, double omega, int sweeps, int project_mean,
                      const void* vel, const void* b, void* w, cudaStream_t st);
void launch_mg_convert_in(int prec, const double* src, void* dst, long long len, cudaStream_t st);
void launch_mg_convert_out(int prec, const void* src, double* dst, long long len,
                           cudaStream_t st);
// bytes per value of the V-cycle's vectors and of its velocity fields
size_t mg_elem_size(int prec);
size_t mg_vel_size(int prec);
// full weighting of a velocity hierarchy (stored as the precision's velocity type)
void launch_mg_restrict_vel(int prec, int dim, const MGLevelDesc& fine, int ncomp, const void* vf,
                            void* vc, cudaStream_t st);

}  // namespace irk
