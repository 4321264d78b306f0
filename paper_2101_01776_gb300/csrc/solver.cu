// Host driver of the Gauss-IRK stage solve and the C ABI (include/irk.h).
//
// One IRK step (Algorithm 1, Sec. 5):
//   k = 0; loop:
//     Y_i, combined fields      k_stage_states           (Eq. stages, Eq. Q0approx)
//     F, rhs = -(Q0^T (x) I) F   k_residual               (Eq. stages, Algorithm 1)
//     stop when ||F|| <= newton_rtol ||F(0)||
//     for the diagonal blocks from last to first:
//       z = rhs_i - sum_{j>i} U_ij dk_hat_j              (Eq. D+U)
//       dk_hat_i = FGMRES(D_i, z, L_P_i)                (Eq. diag_blocks, Eq. Lprec)
//     k += (Q0 R0 (x) I) dk_hat
//   u += dt sum_i b_i k_i                                (Eq. update)
// L_P_i applies one V-cycle for (eta M - dt L_aa) and one for (gamma M - dt L_bb)
// with gamma = gamma* = eta + beta^2/eta (Eq. gamma*) by default.
//
// The Newton-like variant 3 of Sec. 3.2 keeps every d_{k,l} L term inside the
// block upper-triangular pattern of R0 (x) I (exact Newton for s = 2);
// variant 2 keeps only the diagonal terms d_{k,k} L.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "irk_internal.h"

using namespace irk;

namespace {

enum ProfClass {
  P_STAGE = 0, P_RESID, P_STAGEOP, P_UPDATE, P_MG_SMOOTH, P_MG_RESID, P_MG_RESTRICT,
  P_MG_PROLONG, P_MG_COARSE, P_MG_CONVERT, P_MG_SETUP, P_GS_DOT, P_GS_UPDATE, P_REDUCE,
  P_SCALE, P_LINCOMB, P_NORM, P_AXPBY, P_MEAN, P_MG_SMOOTH2, P_POISSON, P_FG_GS1, P_FG_GS2,
  P_FG_NEXT, P_FG_CTL, P_NCLASS
};
const char* kProfNames[P_NCLASS] = {
  "stage_states", "residual", "stage_op", "stage_update", "mg_smooth", "mg_residual",
  "mg_restrict", "mg_prolong", "mg_coarse", "mg_convert", "mg_setup", "gs_multi_dot",
  "gs_update_dot", "reduce", "scale_copy", "lincomb", "norm2", "axpby", "remove_mean",
  "mg_smooth_tile", "poisson_op", "fg_gs1", "fg_gs2", "fg_next", "fg_control"};

struct PendingEvent {
  int cls;
  int a, b;  // indices into the event pool
  double bytes, flops;
};

struct MGLevel {
  MGLevelDesc d;
  void *w, *w2, *b, *r;
  void *w3, *w4;  // Chebyshev iterates on levels that can be the coarsest (l >= 1)
};

}  // namespace

struct irk_handle {
  irk_config cfg;
  HostTableau tab;
  GridDesc g;
  int s = 0, C = 0, dim = 0, npts = 0;
  long long L = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int device = 0;

  char* arena = nullptr;
  size_t arena_bytes = 0, arena_used = 0;
  bool own_arena = true;
  void* ext_arena = nullptr;  // caller-owned arena (irk_create_in)
  size_t ext_bytes = 0;

  double *u = nullptr, *u_save = nullptr, *K = nullptr, *Y = nullptr, *rhs = nullptr,
         *yhat = nullptr, *combos = nullptr, *zbuf = nullptr, *tmp = nullptr, *tmp2 = nullptr;
  double* coef = nullptr;  // coefficient fields of the combined fields in coef_list
  ComboList coef_list = {};
  int coef_slot[IRK_MAX_COMBOS];  // slot in coef of a combined field, or -1
  int ncombo = 0;
  int combo_of[IRK_MAXS][IRK_MAXS];
  double Dq[IRK_MAX_COMBOS * IRK_MAXS];
  int blk_of[IRK_MAXS];

  // FGMRES
  int m = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *partials = nullptr, *dscal = nullptr;
  // fixed staging of the preconditioner: V_j -> prec_in -> L_P -> prec_out -> Z_j
  double *prec_in = nullptr, *prec_out = nullptr;
  // one CUDA graph per diagonal block replaying L_P (valid for graph_dt)
  cudaGraphExec_t gexec[IRK_MAXS] = {};
  double graph_dt = 0.0;
  bool graphs_failed = false;
  int graph_vcycles[IRK_MAXS] = {}, graph_pvcycles[IRK_MAXS] = {};
  long long graph_launches[IRK_MAXS] = {};
  // device-resident FGMRES: one graph per block = coupling + init + WHILE
  // (L_P, matvec, CGS2, Arnoldi) + solution update
  FGState* fgs = nullptr;  // one per block
  cudaStream_t st_aux = nullptr;
  cudaGraphExec_t fgexec[IRK_MAXS] = {};
  double fg_dt = 0.0;
  bool fg_failed = false;
  long long fg_fixed_launches[IRK_MAXS] = {}, fg_body_launches[IRK_MAXS] = {};
  int fg_body_vcycles[IRK_MAXS] = {}, fg_body_pvcycles[IRK_MAXS] = {};
  double fg_seen_its[IRK_MAXS] = {};
  // whole-step graph (Newton loop on the device)
  cudaStream_t st_aux2 = nullptr;
  cudaGraphExec_t stepexec = nullptr;
  double step_dt = 0.0;
  bool step_failed = false;
  long long step_fixed_launches = 0, step_newton_launches = 0;
  double* nws = nullptr;  // Newton state: dscal[400..]
  // exact Newton (variant 4): outer FGMRES on the true stage Jacobian over
  // all s stages; bases Vo ((mo+1) s L), Zo (mo s L), work wo, solution xo,
  // right-hand side fo (= F), JVP scratch jw (= (A0 (x) I) v)
  int mo = 0;
  double *Vo = nullptr, *Zo = nullptr, *wo = nullptr, *xo = nullptr, *fo = nullptr, *jw = nullptr;
  double* hbuf = nullptr;  // pinned host
  int nparts = 0;

  // multigrid
  int prec = 0, nlev = 0, mg_kind = 0;
  size_t esz = 8;
  MGLevel lev[IRK_MAX_LEVELS];
  void* vel[IRK_MAXS][IRK_MAX_LEVELS];
  // FP64 2D advective rows: the four off-diagonal coefficients per level,
  // formed once per Newton iteration from vel (valid for coef_cadv/cdiff)
  bool use_pre = false;
  double* pinv = nullptr;  // 64 x 64 zero-mean pseudo-inverse of -L_h on 8^2 (2D, cdiff = 1)
  void* coefh[IRK_MAXS][IRK_MAX_LEVELS] = {};
  double coef_cadv = 0.0, coef_cdiff = 0.0;
  double mg_omega = 0.8;

  irk_stats stats;
  std::string err;

  // profiling
  std::vector<cudaEvent_t> evpool;
  int ev_used = 0;
  std::vector<PendingEvent> pending;
  irk_kernel_stat prof[P_NCLASS];

  // SDIRK solved stage by stage: a single-stage solver (A = [gamma]) whose
  // arena lies in this handle's arena solves each stage equation in turn;
  // inner_gamma > 0 marks such a single-stage solver
  // Newton starting value (initial_guess = 2): dt of the last accepted step
  // (0: none, -1: stages set by the caller, taken as from a step of the same
  // dt) and the ratio for which the extrapolation matrix sits in dscal[450..]
  double last_dt = 0.0;
  double E_ratio = -2.0;

  irk_handle* inner = nullptr;
  void* inner_arena = nullptr;
  size_t inner_bytes = 0;
  double inner_gamma = 0.0;
};

// creation errors have no handle to live in; one per thread (serving creates handles concurrently)
static thread_local std::string g_create_error;

namespace {

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) {                                                              \
      h->err = std::string("CUDA error: ") + cudaGetErrorString(_e) + " at " #call;       \
      return IRK_ERR_CUDA;                                                                \
    }                                                                                     \
  } while (0)

#define TRY(expr)                   \
  do {                              \
    irk_status _s = (expr);         \
    if (_s != IRK_OK) return _s;    \
  } while (0)

// ---------------------------------------------------------------------------
// profiling: CUDA events around kernel launches on the handle's stream
int prof_begin(irk_handle* h) {
  if (!h->cfg.profile) return -1;
  if (h->ev_used + 2 > (int)h->evpool.size()) return -1;
  int a = h->ev_used++;
  cudaEventRecord(h->evpool[a], h->st);
  return a;
}

void prof_end(irk_handle* h, int a, int cls, double bytes, double flops) {
  if (a < 0) return;
  int b = h->ev_used++;
  cudaEventRecord(h->evpool[b], h->st);
  h->pending.push_back({cls, a, b, bytes, flops});
}

void prof_harvest(irk_handle* h) {
  if (h->pending.empty()) { h->ev_used = 0; return; }
  cudaStreamSynchronize(h->st);
  for (auto& pe : h->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->evpool[pe.a], h->evpool[pe.b]);
    irk_kernel_stat& ks = h->prof[pe.cls];
    ks.launches += 1;
    ks.ms += ms;
    ks.bytes += pe.bytes;
    ks.flops += pe.flops;
  }
  h->pending.clear();
  h->ev_used = 0;
}

void prof_maybe_flush(irk_handle* h) {
  if (h->cfg.profile && h->ev_used + 64 > (int)h->evpool.size()) prof_harvest(h);
}

// Wraps the launch(es) of one kernel class: counts them and, when profiling,
// brackets them with CUDA events and records their algorithmic bytes/flops.
struct ProfScope {
  irk_handle* h;
  int a, cls;
  double bytes, flops;
  ProfScope(irk_handle* h_, int cls_, double bytes_, double flops_, int nlaunch = 1)
      : h(h_), a(-1), cls(cls_), bytes(bytes_), flops(flops_) {
    h->stats.kernel_launches += nlaunch;
    prof_maybe_flush(h);
    a = prof_begin(h);
  }
  ~ProfScope() { prof_end(h, a, cls, bytes, flops); }
};

// FP64 flops per grid point of the operators (counted from the stencils)
double n_flops_per_point(int op) {
  switch (op) {
    case IRK_OP_DIFFUSION_1D: return 5;
    case IRK_OP_BURGERS_1D: return 11;
    case IRK_OP_BURGERS_2D: return 2 * 16;
    default: return 40 + 12 + 6;  // Arakawa + Laplacian + constraint row
  }
}
double jadv_flops_per_point(int op) {
  switch (op) {
    case IRK_OP_DIFFUSION_1D: return 0;
    case IRK_OP_BURGERS_1D: return 4;
    case IRK_OP_BURGERS_2D: return 2 * 12 + 8;
    default: return 2 * 40;
  }
}
double jlin_flops_per_point(int op) {
  switch (op) {
    case IRK_OP_DIFFUSION_1D: case IRK_OP_BURGERS_1D: return 5;
    case IRK_OP_BURGERS_2D: return 2 * 7;
    default: return 7 + 8;
  }
}

// ---------------------------------------------------------------------------
void* arena_take(irk_handle* h, size_t bytes) {
  size_t off = (h->arena_used + 255) & ~(size_t)255;
  if (off + bytes > h->arena_bytes) return nullptr;
  h->arena_used = off + bytes;
  return h->arena + off;
}

irk_status sync_read(irk_handle* h, const double* dsrc, int count) {
  CK(cudaMemcpyAsync(h->hbuf, dsrc, sizeof(double) * count, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

// ||x||_2 of a device vector (blocking)
irk_status dev_norm(irk_handle* h, const double* x, long long len, double* out) {
  const int nb = blas_blocks(len);
  {
    ProfScope ps(h, P_NORM, 8.0 * len, 2.0 * len);
    launch_norm2(x, len, h->partials, h->st);
  }
  {
    ProfScope ps(h, P_REDUCE, 8.0 * nb, nb);
    launch_reduce(h->partials, nb, 1, 1, h->dscal + 200, h->st);
  }
  TRY(sync_read(h, h->dscal + 200, 1));
  *out = std::sqrt(h->hbuf[0]);
  return IRK_OK;
}

// ---------------------------------------------------------------------------
// Row operators of the transformed Jacobian (Eq. D+U, Eq. diag_blocks).
const double* combo_ptr(irk_handle* h, int r, int q) {
  const int idx = h->combo_of[r][q];
  return idx < 0 ? nullptr : h->combos + (long long)idx * h->L;
}

bool keep_coupling(irk_handle* h, int r, int q);

// The advective part of term (r, q): its combined field and, for Burgers-2D,
// the coefficient fields formed from it once per Newton iteration.
void set_combo(irk_handle* h, OpTerm& t, int r, int q) {
  t.combo = keep_coupling(h, r, q) ? combo_ptr(h, r, q) : nullptr;
  const int slot = t.combo ? h->coef_slot[h->combo_of[r][q]] : -1;
  t.coef = (slot >= 0 && h->coef)
               ? h->coef + (long long)slot * combo_coef_fields(h->g.op) * h->npts
               : nullptr;
}

double stage_op_bytes(irk_handle* h, const StageOpArgs& a) {
  double words = 0;
  for (int r = 0; r < a.nrow; ++r) {
    words += h->L * (1 + (a.row[r].base ? 1 : 0));
    for (int t = 0; t < a.row[r].nterm; ++t)
      words += h->L * (1 + (a.row[r].t[t].coef ? combo_coef_fields(h->g.op) / 2.0
                            : a.row[r].t[t].combo ? 1 : 0));
  }
  words += a.copy_len * 2.0;
  return words * 8.0;
}

double stage_op_flops(irk_handle* h, const StageOpArgs& a) {
  double f = 0;
  for (int r = 0; r < a.nrow; ++r)
    for (int t = 0; t < a.row[r].nterm; ++t) {
      const OpTerm& tm = a.row[r].t[t];
      if (tm.coef)  // coefficient form: Burgers-2D 4 coefficients + 2 x (5 FMA, 1 add, 1 mul) + 2 adds;
                    // VSF 16 FMAs (+ the two Laplacians of the linear part)
        f += h->npts * (h->g.op == IRK_OP_VSF_2D ? 34.0 + (tm.lin != 0 ? 24.0 : 0.0) : 30.0);
      else
        f += h->npts * (2.0 * h->C + (tm.combo ? jadv_flops_per_point(h->g.op) : 0) +
                        (tm.lin != 0 ? jlin_flops_per_point(h->g.op) : 0));
    }
  return f;
}

void run_stage_op(irk_handle* h, const StageOpArgs& a) {
  ProfScope ps(h, P_STAGEOP, stage_op_bytes(h, a), stage_op_flops(h, a));
  launch_stage_op(h->g, a, h->st);
}

bool keep_coupling(irk_handle* h, int r, int q) {
  return h->cfg.nonlinear_variant >= 3 || r == q;
}

// y = D_blk x (Eq. diag_blocks); x, y are block vectors of bsize rows of length L
void block_matvec_dt(irk_handle* h, double dt, int blk, const double* x, double* y,
                     const double* copy_src, double* copy_dst) {
  const int a0 = h->tab.bstart[blk], bs = h->tab.bsize[blk], s = h->s;
  StageOpArgs a;
  memset(&a, 0, sizeof(a));
  a.nrow = bs;
  a.dt = dt;
  for (int rr = 0; rr < bs; ++rr) {
    const int r = a0 + rr;
    OpRow& row = a.row[rr];
    row.y = y + (long long)rr * h->L;
    row.sigma = 1;
    for (int qq = 0; qq < bs; ++qq) {
      const int q = a0 + qq;
      OpTerm& t = row.t[row.nterm++];
      t.x = x + (long long)qq * h->L;
      set_combo(h, t, r, q);
      t.m = h->tab.R[r * s + q];
      t.lin = (r == q) ? 1.0 : 0.0;
    }
  }
  a.copy_dst = copy_dst;
  a.copy_src = copy_src;
  a.copy_len = copy_dst ? (long long)bs * h->L : 0;
  run_stage_op(h, a);
}

// z_rows(blk) = rhs_rows(blk) - sum_{l beyond blk} U_{r,l} yhat_l
void upper_coupling(irk_handle* h, double dt, int blk, double* z) {
  const int a0 = h->tab.bstart[blk], bs = h->tab.bsize[blk], s = h->s;
  const int first_later = a0 + bs;
  StageOpArgs a;
  memset(&a, 0, sizeof(a));
  a.nrow = bs;
  a.dt = dt;
  for (int rr = 0; rr < bs; ++rr) {
    const int r = a0 + rr;
    OpRow& row = a.row[rr];
    row.y = z + (long long)rr * h->L;
    row.base = h->rhs + (long long)r * h->L;
    row.alpha = 1;
    row.sigma = -1;
    for (int l = first_later; l < s; ++l) {
      OpTerm& t = row.t[row.nterm++];
      t.x = h->yhat + (long long)l * h->L;
      set_combo(h, t, r, l);
      t.m = h->tab.R[r * s + l];
      t.lin = 0;
    }
  }
  run_stage_op(h, a);
}

// ---------------------------------------------------------------------------
// Multigrid
double mg_level_bytes(irk_handle* h, int l, double fields) {
  return fields * h->lev[l].d.npts * (double)h->esz;
}

// Depth of the V-cycle for shift sigma (the V-cycle-depth autotuning rule).
// The block operators sigma M - dt L are shift dominated: on level l the
// Jacobi diagonal is D_l = sigma + 2 dim cdiff / h_l^2, and once sigma >= D_l/2
// damped Jacobi alone reduces every error mode by at least (1 - omega/2) per
// sweep, so coarsening further buys nothing.  The cycle stops at the first
// such level (never above level 1: at least one coarse correction), or at the
// bottom of the hierarchy for an unshifted operator (the Poisson block).
int mg_depth(irk_handle* h, double sigma, double cdiff) {
  if (h->cfg.mg_levels > 0) return std::min(h->cfg.mg_levels, h->nlev);
  if (!(sigma > 0)) return h->nlev;
  for (int l = 1; l < h->nlev; ++l) {
    const double hl = h->lev[l].d.h;
    const double D = sigma + 2.0 * h->dim * cdiff / (hl * hl);
    if (sigma >= 0.5 * D) return l + 1;
  }
  return h->nlev;
}

// Shift of block row r in L_P: eta on the first row of a block, gamma (gamma*
// or eta) on the second (Eq. Lprec, Eq. gamma*).
double row_shift(irk_handle* h, int r) {
  const int blk = h->blk_of[r];
  if (r == h->tab.bstart[blk]) return h->tab.eta[blk];
  return (h->cfg.gamma_mode == 1) ? h->tab.eta[blk] : h->tab.gamma_star[blk];
}

// Coefficient (velocity) hierarchy of every diagonal row from its combined
// field (k,k), restricted down to the depth that row's V-cycle reaches.
void mg_setup(irk_handle* h, double dt) {
  if (h->g.op == IRK_OP_DIFFUSION_1D) return;
  for (int k = 0; k < h->s; ++k) {
    const int depth = mg_depth(h, row_shift(h, k), dt * h->g.nu);
    // FP64 Burgers-2D rows: the two finest levels' velocity and coefficients
    // in one launch (the same values as the separate kernels below)
    const bool fused = h->g.op == IRK_OP_BURGERS_2D && h->use_pre && depth >= 2;
    if (fused) {
      const double n0 = h->lev[0].d.npts;
      ProfScope ps(h, P_MG_SETUP, 8.0 * (2.0 + 6.0 + 6.0 / 4.0) * n0, 4.0 * n0 * 1.25 + 5.0 * n0);
      launch_mg_setup2(h->lev[0].d, h->lev[1].d, dt, dt * h->g.nu, combo_ptr(h, k, k),
                       h->vel[k][0], h->coefh[k][0], h->vel[k][1], h->coefh[k][1], h->st);
    } else {
      ProfScope ps(h, P_MG_SETUP, 8.0 * h->L + mg_level_bytes(h, 0, h->dim), 0);
      launch_velocity_from_combo(h->g, combo_ptr(h, k, k), h->vel[k][0], h->prec, h->st);
    }
    for (int l = fused ? 1 : 0; l + 1 < depth; ++l) {
      ProfScope ps(h, P_MG_SETUP,
                   mg_level_bytes(h, l, h->dim) * 1.25 * mg_vel_size(h->prec) / h->esz, 0);
      launch_mg_restrict_vel(h->prec, h->dim, h->lev[l].d, h->dim, h->vel[k][l], h->vel[k][l + 1],
                             h->st);
    }
    if (h->use_pre)
      for (int l = fused ? 2 : 0; l < depth; ++l) {
        ProfScope ps(h, P_MG_SETUP, mg_level_bytes(h, l, 6.0), 4.0 * h->lev[l].d.npts);
        launch_mg_coef(h->prec, h->lev[l].d, dt, dt * h->g.nu, h->vel[k][l], h->coefh[k][l],
                       h->st);
      }
  }
  h->coef_cadv = dt;
  h->coef_cdiff = dt * h->g.nu;
}

// FP64 operations (an FMA counts 2) per point of the MG kernels as built:
// per component a sweep takes one FMA per neighbour, the diagonal FMA and
// the (1 - omega) product; the residual one FMA per neighbour and the
// diagonal FMA.  Coefficients formed on the fly cost one FMA per neighbour
// and point (shared by the components); precomputed ones (MG_ADVECTIVE_PRE)
// and the constant diffusion stencil cost nothing per sweep.
double mg_coef_flops(int kind, int dim) {
  if (kind == MG_ADVECTIVE) return 4.0 * dim;
  if (kind == MG_CONSERVATIVE_1D) return 4.0;
  return 0.0;
}
double mg_sweep_flops(int kind, int dim, int ncomp) {
  return ncomp * (4.0 * dim + 3.0) + mg_coef_flops(kind, dim);
}
double mg_resid_flops(int kind, int dim, int ncomp) {
  return ncomp * (4.0 * dim + 2.0) + mg_coef_flops(kind, dim);
}

// `sweeps` damped-Jacobi sweeps on level l (from w = 0 when from_zero); the
// iterate ends in cur (cur/alt swap as the sweeps ping-pong), or in `last`
// when given (the caller's output buffer).  Pairs of sweeps go to the
// temporally blocked two-sweep kernel where it pays; it reads b on a halo, so
// it never writes into b.
// A pointwise epilogue for the last sweep of a V-cycle in FP64 storage:
// out = bcoef * base + coef * w (a pointwise coupling row of L_P).
struct MGEpilogue {
  double* out;
  const double* base;
  double coef;         // out = bcoef * base + coef * w
  double bcoef = 1.0;
};

// b64 / out64: a reduced-precision finest level reading its right-hand side
// from the FP64 input and writing its last sweep to the FP64 output (single
// sweeps only: the callers pass them with one sweep)
bool jacobi_sweeps(irk_handle* h, int l, int kind, int ncomp, double sigma, double cadv,
                   double cdiff, double om, const void* vel, const void* b, int sweeps,
                   bool from_zero, void*& cur, void*& alt, void* last,
                   const MGEpilogue* epi = nullptr, const double* b64 = nullptr,
                   double* out64 = nullptr) {
  bool epi_done = false;
  const MGLevelDesc& d = h->lev[l].d;
  const int prec = h->prec, dim = h->dim;
  // velocity fields, in units of the vectors' value size (BF16 velocities: half)
  const double velf = ((kind == MG_DIFFUSION) ? 0
                       : (kind == MG_ADVECTIVE_PRE) ? 4 : (kind == MG_CONSERVATIVE_1D ? 1 : dim)) *
                      (kind == MG_ADVECTIVE_PRE ? 1.0 : (double)mg_vel_size(prec) / h->esz);
  // one sweep; the tile kernels' undamped sweeps (1 - omega = 0) skip the
  // damping product and the add of the diagonal FMA: 2 flops less per value
  const double fsw = mg_sweep_flops(kind, dim, ncomp) * d.npts;
  const double fsw_tile = (om == 1.0 ? fsw - 2.0 * ncomp * d.npts : fsw);
  const double f0 = (double)ncomp * d.npts;                       // a sweep from zero
  const double pts = (double)ncomp * d.npts;
  int sw = 0;
  while (sw < sweeps) {
    // a first sweep from zero reads no w, so it may write in place
    const int first = from_zero && sw == 0;
    void* dst = first ? cur : alt;
    const bool ends_pair = (sw + 2 == sweeps);
    const int rem = sweeps - sw;
    // three sweeps per launch for 3, 5, 6, 7, ... remaining (4 go as two pairs)
    if (rem >= 3 && rem != 4 && mg_smooth3_pays(prec, dim, d) && !(rem == 3 && last == b)) {
      if (rem == 3 && last) dst = last;
      ProfScope ps(h, P_MG_SMOOTH2, mg_level_bytes(h, l, (first ? 2.0 : 3.0) * ncomp + velf),
                   first ? f0 + 2.0 * fsw_tile : 3.0 * fsw_tile);
      launch_mg_smooth3(prec, kind, d, ncomp, sigma, cadv, cdiff, om, vel, b, cur, dst, first,
                        h->st, h->cfg.mg_tile_rows);
      sw += 3;
    } else if (sw + 1 < sweeps && mg_smooth2_pays(prec, dim, kind, d, first) && !(ends_pair && last == b)) {
      if (ends_pair && last) dst = last;
      ProfScope ps(h, P_MG_SMOOTH2, mg_level_bytes(h, l, (first ? 2.0 : 3.0) * ncomp + velf),
                   first ? f0 + fsw_tile : 2.0 * fsw_tile);
      launch_mg_smooth2(prec, kind, d, ncomp, sigma, cadv, cdiff, om, vel, b, cur, dst, first,
                        h->st);
      sw += 2;
    } else {
      const bool final = (sw + 1 == sweeps);
      if (final && last) dst = last;
      const bool wide = final && out64 && prec != IRK_MG_FP64;
      const bool with_epi = final && epi && !first && ((last && prec == IRK_MG_FP64) || wide);
      // b and the result in FP64 instead of the storage type
      const double wide_bytes = (b64 ? (8.0 - h->esz) * ncomp * d.npts : 0.0) +
                                (wide ? (8.0 - h->esz) * ncomp * d.npts : 0.0);
      ProfScope ps(h, P_MG_SMOOTH, mg_level_bytes(h, l, first ? 2.0 * ncomp : 3.0 * ncomp + velf) +
                                       wide_bytes + (with_epi ? 16.0 * ncomp * d.npts : 0.0),
                   (first ? f0 : fsw) + (with_epi ? 2.0 * ncomp * d.npts : 0.0));
      launch_mg_smooth(prec, dim, kind, d, ncomp, sigma, cadv, cdiff, om, vel, b, cur, dst, first,
                       h->st, with_epi ? epi->out : nullptr, with_epi ? epi->base : nullptr,
                       with_epi ? epi->coef : 0.0, with_epi ? epi->bcoef : 1.0, b64,
                       wide ? out64 : nullptr);
      epi_done = epi_done || with_epi;
      sw += 1;
    }
    if (dst == alt) std::swap(cur, alt);
  }
  return epi_done;
}

// One V-cycle for A = sigma I + cadv adv(vel_k) - cdiff L on ncomp fields.
// in/out: double, ncomp * npts_fine.  In FP64 storage the input is read in
// place and the last fine-level sweep writes the output directly.
// Returns whether `epi` (if given) was applied by the last fine-level sweep.
bool vcycle(irk_handle* h, int row, int kind, int ncomp, double sigma, double cadv, double cdiff,
            int project_mean, const double* in, double* out, const MGEpilogue* epi = nullptr) {
  TraceRange tr("vcycle");
  bool epi_done = false;
  const int nl = mg_depth(h, sigma, cdiff), prec = h->prec, dim = h->dim;
  const double om = h->mg_omega;
  // shift-dominated rows of 2D grids (sigma >= 0.15 D on the finest level)
  // take mg_shifted_sweeps pre- and post-sweeps: measured on 2D Burgers and
  // the VSF vorticity rows, their Krylov counts do not drop with more
  // smoothing (on the 1D grids they do, so 1D keeps mg_pre/mg_post)
  int npre = h->cfg.mg_pre, post = h->cfg.mg_post;
  {
    const double h0 = h->lev[0].d.h;
    const double D0 = sigma + 2.0 * dim * cdiff / (h0 * h0);
    if (dim == 2 && h->cfg.mg_shifted_sweeps > 0 && sigma >= 0.15 * D0)
      npre = post = h->cfg.mg_shifted_sweeps;
  }
  const void* vrow[IRK_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) vrow[l] = (row >= 0) ? h->vel[row][l] : nullptr;
  // FP64 2D advective rows read the precomputed coefficients (kind kk, crow);
  // the one-CTA coarsest solve keeps the velocity form (kind, vrow)
  const bool pre = h->use_pre && kind == MG_ADVECTIVE && row >= 0 && cadv == h->coef_cadv &&
                   cdiff == h->coef_cdiff;
  const int kk = pre ? MG_ADVECTIVE_PRE : kind;
  const void* crow[IRK_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) crow[l] = pre ? h->coefh[row][l] : vrow[l];
  const long long n0 = (long long)ncomp * h->lev[0].d.npts;
  const bool alias = (prec == IRK_MG_FP64);
  const double velf = ((kk == MG_DIFFUSION) ? 0
                       : (kk == MG_ADVECTIVE_PRE) ? 4 : (kk == MG_CONSERVATIVE_1D ? 1 : dim)) *
                      (kk == MG_ADVECTIVE_PRE ? 1.0 : (double)mg_vel_size(prec) / h->esz);
  const double fsweep = mg_sweep_flops(kk, dim, ncomp), fresid = mg_resid_flops(kk, dim, ncomp);
  // a single pre-sweep starts from zero (w = dinv b): it is folded into the
  // residual and rebuilt by the prolongation, one launch less per level
  const bool fold_pre = (npre == 1);
  // deep periodic Poisson cycles: the levels from 32^2 down run in one CTA
  // with an exact zero-mean solve on 8^2
  int lb = nl;
  if (dim == 2 && kind == MG_DIFFUSION && sigma == 0.0 && ncomp == 1 && project_mean && h->pinv &&
      h->lev[nl - 1].d.n == 8) {
    lb = nl - 1;
    while (lb > 0 && h->lev[lb - 1].d.n <= 32) --lb;
  }
  // reduced-precision storage with the folded pre-sweep and one post-sweep:
  // the finest level's three kernels read b from the FP64 input and the last
  // sweep writes the FP64 output, so no conversion launches are needed
  const bool wide_io = !alias && fold_pre && post == 1 && nl >= 2 && lb >= 1;
  const double* b64 = wide_io ? in : nullptr;
  const void* bl[IRK_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) bl[l] = h->lev[l].b;
  if (alias) {
    bl[0] = in;
  } else if (!wide_io) {
    ProfScope ps(h, P_MG_CONVERT, n0 * (8.0 + h->esz), 0);
    launch_mg_convert_in(prec, in, h->lev[0].b, n0, h->st);
  }
  void* cur[IRK_MAX_LEVELS];
  void* alt[IRK_MAX_LEVELS];
  for (int l = 0; l + 1 < nl && l < lb; ++l) {
    MGLevel& lv = h->lev[l];
    cur[l] = lv.w;
    alt[l] = lv.w2;
    const int fuse_mode = h->cfg.mg_fuse_transfer ? h->cfg.mg_fuse_transfer
                                                  : (prec == IRK_MG_FP64 ? 2 : 1);
    if (fold_pre && dim == 2 && lv.d.n >= 32 && ncomp <= 2 && fuse_mode == 1) {
      // residual and restriction in one launch: r stays on chip
      const double wb = (l == 0 && b64) ? (8.0 - h->esz) * ncomp * lv.d.npts : 0.0;
      ProfScope ps(h, P_MG_RESID, mg_level_bytes(h, l, ncomp * 1.25 + velf) + wb,
                   (fresid + 2.0 * ncomp) * lv.d.npts + 12.0 * ncomp * lv.d.npts / 4);
      launch_mg_resid0_restrict(prec, kk, lv.d, ncomp, sigma, cadv, cdiff, om, crow[l], bl[l],
                                h->lev[l + 1].b, h->st, l == 0 ? b64 : nullptr);
      continue;
    }
    if (fold_pre) {
      const double wb = (l == 0 && b64) ? (8.0 - h->esz) * ncomp * lv.d.npts : 0.0;
      ProfScope ps(h, P_MG_RESID, mg_level_bytes(h, l, 2.0 * ncomp + velf) + wb,
                   (fresid + 2.0 * ncomp) * lv.d.npts);
      launch_mg_residual0(prec, dim, kk, lv.d, ncomp, sigma, cadv, cdiff, om, crow[l], bl[l],
                          lv.r, h->st, l == 0 ? b64 : nullptr);
    } else {
      jacobi_sweeps(h, l, kk, ncomp, sigma, cadv, cdiff, om, crow[l], bl[l], npre, true,
                    cur[l], alt[l], nullptr);
      ProfScope ps(h, P_MG_RESID, mg_level_bytes(h, l, 3.0 * ncomp + velf),
                   fresid * lv.d.npts);
      launch_mg_residual(prec, dim, kk, lv.d, ncomp, sigma, cadv, cdiff, crow[l], bl[l], cur[l],
                         lv.r, h->st);
    }
    {
      ProfScope ps(h, P_MG_RESTRICT, mg_level_bytes(h, l, ncomp) * (1.0 + 1.0 / (1 << dim)),
                   (double)ncomp * lv.d.npts / (1 << dim) * (dim == 1 ? 4 : 12));
      launch_mg_restrict(prec, dim, lv.d, ncomp, lv.r, h->lev[l + 1].b, h->st);
    }
  }
  if (lb < nl) {
    MGLevel& lv = h->lev[lb];
    double words = 0;
    for (int l = lb; l < nl; ++l) words += 2.0 * h->lev[l].d.npts;
    ProfScope ps(h, P_MG_COARSE, words * h->esz,
                 (npre + post + 1) * 7.0 * lv.d.npts * 4.0 / 3.0 + 2.0 * 64 * 64);
    launch_mg_bottom(prec, lv.d, cdiff, om, npre, post, h->pinv, bl[lb], lv.w, h->st);
    cur[lb] = lv.w;
  } else {
    const int c = nl - 1;
    MGLevel& lc = h->lev[c];
    if (lc.d.npts <= 256) {
      ProfScope ps(h, P_MG_COARSE, mg_level_bytes(h, c, 2.0 * ncomp + (kind == MG_DIFFUSION ? 0 : dim)),
                   mg_sweep_flops(kind, dim, ncomp) * lc.d.npts * h->cfg.mg_coarse_sweeps);
      launch_mg_coarse(prec, dim, kind, lc.d, ncomp, sigma, cadv, cdiff, om,
                       h->cfg.mg_coarse_sweeps, project_mean, vrow[c], bl[c], lc.w, h->st);
      cur[c] = lc.w;
    } else {
      // shift-dominated coarsest level (sigma >= D/2): undamped Jacobi, whose
      // iteration matrix has norm <= 1 - sigma/D <= 1/2 there, swept to a
      // the target reduction (mg_coarse_reduction, default 2e-2), 2..12 sweeps
      const double hc = lc.d.h;
      const double D = sigma + 2.0 * dim * cdiff / (hc * hc);
      const double omc = (sigma >= 0.5 * D) ? 1.0 : om;
      const double rho = 1.0 - omc * sigma / D;
      const double red = h->cfg.mg_coarse_reduction > 0 ? h->cfg.mg_coarse_reduction : 2e-2;
      int sweeps = (rho > 0 && rho < 1) ? (int)std::ceil(std::log(red) / std::log(rho)) : 2;
      sweeps = std::max(2, std::min(sweeps, 12));
      cur[c] = lc.w;
      alt[c] = lc.w2;
      const double rhoj = 1.0 - sigma / D;  // undamped Jacobi on [sigma/D, 2 - sigma/D]
      int msteps = 0;
      const bool smem_ok = (omc == 1.0 && dim == 2 && lc.d.n >= 32 && rhoj > 0 && rhoj < 1);
      int gs_sweeps = 0;
      if (h->cfg.mg_coarse_smoother == 2 && smem_ok) {
        // red-black Gauss-Seidel: rho_GS = rho_J^2 for the consistently
        // ordered 5-point stencil
        gs_sweeps = (int)std::ceil(std::log(red) / (2.0 * std::log(rhoj)));
        gs_sweeps = std::max(1, std::min(gs_sweeps, 6));
      }
      if (h->cfg.mg_coarse_smoother == 1 && smem_ok && lc.w3) {
        // Chebyshev acceleration: the error after m steps is at most
        // 1/T_m(1/rho); the smallest even m in 2..12 reaching the target
        const double ach = std::acosh(1.0 / rhoj);
        for (int m = 2; m <= 12; m += 2)
          if (1.0 / std::cosh(m * ach) <= red) { msteps = m; break; }
        if (msteps == 0) msteps = 12;
      }
      if (gs_sweeps > 0) {
        void* src = lc.w;
        void* dst = lc.w2;
        for (int q = 0; q < gs_sweeps; ++q) {
          const int first = (q == 0);
          ProfScope ps(h, P_MG_SMOOTH2, mg_level_bytes(h, c, (first ? 2.0 : 3.0) * ncomp + velf),
                       (first ? 0.5 * ncomp + 0.5 * fsweep : fsweep) * lc.d.npts);
          launch_mg_rbgs(prec, kk, lc.d, ncomp, sigma, cadv, cdiff, crow[c], bl[c], src, dst, first,
                         h->st);
          std::swap(src, dst);
        }
        cur[c] = src;
      } else if (msteps > 0 && msteps < sweeps) {
        // three-term weights: w_1 = 1, w_2 = 1/(1 - rho^2/2), w_{k+1} = 1/(1 - rho^2 w_k/4)
        double wk[13];
        wk[1] = 1.0;
        wk[2] = 1.0 / (1.0 - 0.5 * rhoj * rhoj);
        for (int q = 3; q <= msteps; ++q) wk[q] = 1.0 / (1.0 - 0.25 * rhoj * rhoj * wk[q - 1]);
        void* bufA[2] = {lc.w, lc.w2};
        void* bufB[2] = {lc.w3, lc.w4};
        void** in = bufB;   // (x_{k-1}, x_k) of the previous pair
        void** outp = bufA;
        for (int q = 0; q < msteps; q += 2) {
          const int first = (q == 0);
          ProfScope ps(h, P_MG_SMOOTH2, mg_level_bytes(h, c, (first ? 3.0 : 5.0) * ncomp + velf),
                       (first ? ncomp + fsweep : 2.0 * fsweep + 6.0 * ncomp) * lc.d.npts);
          launch_mg_cheb2(prec, kk, lc.d, ncomp, sigma, cadv, cdiff, crow[c], bl[c], in[0], in[1],
                          outp[0], outp[1], wk[q + 1], wk[q + 2], first, h->st);
          std::swap(in, outp);
        }
        cur[c] = in[1];  // x_m
      } else {
        jacobi_sweeps(h, c, kk, ncomp, sigma, cadv, cdiff, omc, crow[c], bl[c], sweeps, true,
                      cur[c], alt[c], nullptr);
      }
    }
  }
  bool wrote_out = false;
  for (int l = std::min(nl, lb) - 2 + (lb < nl ? 1 : 0); l >= 0; --l) {
    MGLevel& lv = h->lev[l];
    {
      const double wb = (l == 0 && b64) ? (8.0 - h->esz) * ncomp * lv.d.npts : 0.0;
      ProfScope ps(h, P_MG_PROLONG, mg_level_bytes(h, l, 2.0 * ncomp + (double)ncomp / (1 << dim)) + wb,
                   (double)ncomp * lv.d.npts * 3);
      if (fold_pre)
        launch_mg_prolong_set(prec, dim, lv.d, ncomp, sigma, cadv, cdiff, om, bl[l], cur[l + 1],
                              cur[l], h->st, l == 0 ? b64 : nullptr);
      else
        launch_mg_prolong_add(prec, dim, lv.d, ncomp, cur[l + 1], cur[l], h->st);
    }
    if (post > 0) {
      const bool to_out = (alias || wide_io) && l == 0;
      const bool e = jacobi_sweeps(h, l, kk, ncomp, sigma, cadv, cdiff, om, crow[l], bl[l], post,
                                   false, cur[l], alt[l], (to_out && alias) ? (void*)out : nullptr,
                                   to_out ? epi : nullptr, l == 0 ? b64 : nullptr,
                                   (to_out && wide_io) ? out : nullptr);
      epi_done = epi_done || e;
      if (to_out) wrote_out = true;
    }
  }
  if (!wrote_out) {
    ProfScope ps(h, P_MG_CONVERT, n0 * (8.0 + h->esz), 0);
    launch_mg_convert_out(prec, cur[0], out, n0, h->st);
  }
  h->stats.vcycles += 1;
  if (row < 0 && kind == MG_DIFFUSION) h->stats.poisson_vcycles += 1;
  return epi_done;
}

// Inner inverse (sigma M - dt L_kk)^{-1} of one block row, approximated by MG.
bool row_prec(irk_handle* h, double dt, int row, double sigma, const double* in, double* out,
              const MGEpilogue* epi = nullptr) {
  const int op = h->g.op;
  if (op == IRK_OP_VSF_2D) {
    // Picard-type lower-triangular solve of the (omega, psi) row (Eq. vsf-system-1):
    // omega: sigma - dt (J_A(psibar, .) + nu L); psi: (-L) z_psi = z_omega - r_psi / dt
    // the psi right-hand side z_omega - r_psi / dt is pointwise: written by
    // the last sweep of the omega V-cycle when it can be, else two axpby
    const MGEpilogue ep = {h->tmp2, in + h->npts, 1.0, -1.0 / dt};
    if (!vcycle(h, row, MG_ADVECTIVE, 1, sigma, dt, dt * h->g.nu, 0, in, out, &ep)) {
      ProfScope ps(h, P_AXPBY, 40.0 * h->npts, 3.0 * h->npts, 2);
      launch_axpby(h->tmp2, 1.0, out, 0.0, h->npts, h->st);
      launch_axpby(h->tmp2, -1.0 / dt, in + h->npts, 1.0, h->npts, h->st);
    }
    vcycle(h, -1, MG_DIFFUSION, 1, 0.0, 0.0, 1.0, 1, h->tmp2, out + h->npts);
    return false;
  }
  const int kind = (op == IRK_OP_BURGERS_1D) ? MG_CONSERVATIVE_1D
                   : (op == IRK_OP_BURGERS_2D) ? MG_ADVECTIVE : MG_DIFFUSION;
  return vcycle(h, row, kind, h->C, sigma, dt, dt * h->g.nu, 0, in, out, epi);
}

// z = L_P(v) for block blk (Eq. Lprec with the (2,1) block of Eq. diag_blocks)
void block_prec(irk_handle* h, double dt, int blk, const double* v, double* z) {
  const int a = h->tab.bstart[blk], bs = h->tab.bsize[blk], s = h->s;
  const double eta = h->tab.eta[blk];
  if (bs == 1) {
    row_prec(h, dt, a, eta, v, z);
    return;
  }
  const int b = a + 1;
  const double gamma = (h->cfg.gamma_mode == 1) ? eta : h->tab.gamma_star[blk];
  // a mass-only coupling row (no advective part for (b, a)) is pointwise:
  // r_b' = v_b - R0_ba z_a is written by the last sweep of the first V-cycle
  OpTerm probe;
  memset(&probe, 0, sizeof(probe));
  set_combo(h, probe, b, a);
  if (!probe.combo) {
    const MGEpilogue epi = {h->tmp, v + h->L, -h->tab.R[b * s + a], 1.0};
    if (row_prec(h, dt, a, eta, v, z, &epi)) {
      row_prec(h, dt, b, gamma, h->tmp, z + h->L);
      return;
    }
  } else {
    row_prec(h, dt, a, eta, v, z);
  }
  StageOpArgs op;
  memset(&op, 0, sizeof(op));
  op.nrow = 1;
  op.dt = dt;
  OpRow& row = op.row[0];
  row.y = h->tmp;
  row.base = v + h->L;
  row.alpha = 1;
  row.sigma = -1;
  row.nterm = 1;
  row.t[0].x = z;
  set_combo(h, row.t[0], b, a);
  row.t[0].m = h->tab.R[b * s + a];
  row.t[0].lin = 0;
  run_stage_op(h, op);
  row_prec(h, dt, b, gamma, h->tmp, z + h->L);
}

// ---------------------------------------------------------------------------
// L_P of block blk from prec_in to prec_out.  Its launch sequence is fixed
// for a given dt (the V-cycle depth, shifts and buffers do not change), so it
// is captured once into a CUDA graph per block and replayed; a capture that
// the stream does not allow (e.g. the legacy default stream) falls back to
// direct launches of the same kernels.
void drop_graphs(irk_handle* h) {
  for (int k = 0; k < IRK_MAXS; ++k)
    if (h->gexec[k]) {
      cudaGraphExecDestroy(h->gexec[k]);
      h->gexec[k] = nullptr;
    }
}

irk_status apply_prec(irk_handle* h, double dt, int blk) {
  const bool want = h->cfg.use_graphs && !h->cfg.profile && !h->graphs_failed;
  if (want && h->graph_dt != dt) {
    drop_graphs(h);
    h->graph_dt = dt;
  }
  if (want && !h->gexec[blk]) {
    const irk_stats saved = h->stats;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      block_prec(h, dt, blk, h->prec_in, h->prec_out);
      e = cudaStreamEndCapture(h->st, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[blk], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    h->graph_vcycles[blk] = h->stats.vcycles - saved.vcycles;
    h->graph_pvcycles[blk] = h->stats.poisson_vcycles - saved.poisson_vcycles;
    h->graph_launches[blk] = h->stats.kernel_launches - saved.kernel_launches;
    h->stats = saved;
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->gexec[blk] = nullptr;
      h->graphs_failed = true;
    }
  }
  if (want && h->gexec[blk]) {
    CK(cudaGraphLaunch(h->gexec[blk], h->st));
    h->stats.vcycles += h->graph_vcycles[blk];
    h->stats.poisson_vcycles += h->graph_pvcycles[blk];
    h->stats.kernel_launches += h->graph_launches[blk];
    return IRK_OK;
  }
  block_prec(h, dt, blk, h->prec_in, h->prec_out);
  return IRK_OK;
}

// Flexible GMRES(m), right preconditioned, classical Gram-Schmidt applied
// twice (step a8), on vectors of length Lb with bases V ((m+1) Lb) and
// Z (m Lb) and the work vector w.  step(j) leaves Z_j = P_j^{-1} V_j and
// w = A Z_j (P_j may change with j); apply(x, y) computes y = A x for
// restarts; counted() runs once per iteration.  V_j is also written to
// `stage` when given (the fixed input buffer of a captured preconditioner).
template <class Step, class Apply, class Counted>
irk_status fgmres_core(irk_handle* h, long long Lb, int m, int maxit, double* V, double* Z,
                       double* w, double* stage, const double* b, double* x, double rtol,
                       int* its_out, double* relres_out, Step step, Apply apply, Counted counted) {
  const long long ldv = Lb;
  double beta;
  TRY(dev_norm(h, b, Lb, &beta));
  CK(cudaMemsetAsync(x, 0, sizeof(double) * Lb, h->st));
  *its_out = 0;
  *relres_out = 0;
  if (!(beta > 0)) {
    if (!std::isfinite(beta)) { h->err = "non-finite right-hand side in FGMRES"; return IRK_ERR_NEWTON_DIVERGED; }
    return IRK_OK;
  }
  const double target = rtol * beta;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  const double* r = b;
  double rnorm = beta;
  int total = 0;
  const int nb = blas_blocks(Lb);
  double* dh1 = h->dscal;        // [0, 64)
  double* dh2 = h->dscal + 64;   // [64, 129)
  double* dnr = h->dscal + 130;  // [130]
  while (true) {
    {
      ProfScope ps(h, P_SCALE, 16.0 * Lb, (double)Lb);
      launch_scale_copy(r, 1.0 / rnorm, V, stage, Lb, h->st);
    }
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = rnorm;
    int jlast = -1;
    double res = rnorm;
    for (int j = 0; j < m; ++j) {
      TRY(step(j));  // Z_j = P^{-1} V_j, w = A Z_j
      const int nv = j + 1;
      {
        ProfScope ps(h, P_GS_DOT, 8.0 * Lb * (nv + 1), 2.0 * Lb * nv);
        launch_multi_dot(V, ldv, nv, w, Lb, h->partials, h->st);
      }
      {
        ProfScope ps(h, P_REDUCE, 8.0 * nb * nv, (double)nb * nv);
        launch_reduce(h->partials, nb, nv, nv, dh1, h->st);
      }
      {
        ProfScope ps(h, P_GS_UPDATE, 8.0 * Lb * (nv + 2), 4.0 * Lb * nv + 2.0 * Lb);
        launch_update_dot(V, ldv, nv, dh1, w, Lb, 1, h->partials, h->st);
      }
      {
        ProfScope ps(h, P_REDUCE, 8.0 * nb * (nv + 1), (double)nb * (nv + 1));
        launch_reduce(h->partials, nb, nv + 1, nv, dh2, h->st);
      }
      {
        ProfScope ps(h, P_GS_UPDATE, 8.0 * Lb * (nv + 2), 2.0 * Lb * nv + 2.0 * Lb);
        launch_update_dot(V, ldv, nv, dh2, w, Lb, 0, h->partials, h->st);
      }
      {
        ProfScope ps(h, P_REDUCE, 8.0 * nb, (double)nb);
        launch_reduce(h->partials + nv, nb, nv + 1, 1, dnr, h->st);
      }
      CK(cudaMemcpyAsync(h->hbuf, h->dscal, sizeof(double) * 131, cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      const double* hh1 = h->hbuf;
      const double* hh2 = h->hbuf + 64;
      const double nrm2 = h->hbuf[130];
      for (int i = 0; i < nv; ++i) H[i * m + j] = hh1[i] + hh2[i];
      const double hn = std::sqrt(std::max(nrm2, 0.0));
      if (!std::isfinite(hn)) { h->err = "non-finite Krylov vector"; return IRK_ERR_KRYLOV_BREAKDOWN; }
      // apply the previous rotations to column j, then a new one
      for (int i = 0; i < j; ++i) {
        const double t0 = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        const double t1 = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t0;
        H[(i + 1) * m + j] = t1;
      }
      const double hjj = H[j * m + j];
      const double den = std::hypot(hjj, hn);
      cs[j] = den > 0 ? hjj / den : 1.0;
      sn[j] = den > 0 ? hn / den : 0.0;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      res = std::fabs(gv[j + 1]);
      ++total;
      jlast = j;
      counted();
      if (res <= target || hn <= 1e-300 || total >= maxit) break;
      {
        ProfScope ps(h, P_SCALE, 16.0 * Lb, (double)Lb);
        launch_scale_copy(w, 1.0 / hn, V + (long long)(j + 1) * ldv, stage, Lb, h->st);
      }
    }
    // y = H^{-1} g on the leading (jlast+1) block, x += Z y
    const int k = jlast + 1;
    for (int i = k - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int q = i + 1; q < k; ++q) acc -= H[i * m + q] * y[q];
      y[i] = acc / H[i * m + i];
    }
    {
      ProfScope ps(h, P_LINCOMB, 8.0 * Lb * (k + 2), 2.0 * Lb * k);
      launch_lincomb(x, Z, ldv, k, y.data(), Lb, h->st);
    }
    *its_out = total;
    if (res <= target) { *relres_out = res / beta; return IRK_OK; }
    if (total >= maxit) { *relres_out = res / beta; return IRK_OK; }
    // restart: r = b - A x
    apply(x, w);
    {
      ProfScope ps(h, P_AXPBY, 24.0 * Lb, 2.0 * Lb);
      launch_axpby(w, 1.0, b, -1.0, Lb, h->st);
    }
    r = w;
    TRY(dev_norm(h, r, Lb, &rnorm));
    if (!(rnorm > 0)) return IRK_OK;
  }
}

// FGMRES on diagonal block blk of Algorithm 1 (step a8), preconditioned by L_P.
irk_status fgmres(irk_handle* h, double dt, int blk, const double* b, double* x, double rtol,
                  int* its_out, double* relres_out) {
  const int bs = h->tab.bsize[blk];
  const long long Lb = (long long)bs * h->L;
  auto step = [&](int j) -> irk_status {
    TRY(apply_prec(h, dt, blk));  // prec_in (= V_j) -> prec_out
    // w = D z_j, and Z_j = z_j
    block_matvec_dt(h, dt, blk, h->prec_out, h->w, h->prec_out, h->Z + (long long)j * Lb);
    return IRK_OK;
  };
  auto apply = [&](const double* xin, double* y) { block_matvec_dt(h, dt, blk, xin, y, nullptr, nullptr); };
  auto counted = [&]() {
    h->stats.krylov_its += 1;
    h->stats.prec_apps += bs;
  };
  return fgmres_core(h, Lb, h->m, h->cfg.krylov_maxit, h->V, h->Z, h->w, h->prec_in, b, x, rtol,
                     its_out, relres_out, step, apply, counted);
}

// ---------------------------------------------------------------------------
void set_stage_args(irk_handle* h, StageStateArgs& a, double dt, const double* u,
                    const double* K, double* Y, double* combos) {
  memset(&a, 0, sizeof(a));
  a.s = h->s;
  a.ncombo = combos ? h->ncombo : 0;
  a.L = h->L;
  a.dt = dt;
  for (int i = 0; i < h->s * h->s; ++i) a.A[i] = h->tab.A[i];
  for (int i = 0; i < h->ncombo * h->s; ++i) a.D[i] = h->Dq[i];
  a.u = u;
  a.K = K;
  a.Y = Y;
  a.combos = combos;
}

// stage states + residual + ||F|| (blocking read of the norm)
// Stage states, residual and ||F||^2 (to dscal[201]); launches only.
void launch_eval_residual(irk_handle* h, double t_n, double dt, const double* K, double* rhs,
                          double* Fraw, bool combos) {
  StageStateArgs sa;
  set_stage_args(h, sa, dt, h->u, K, h->Y, combos ? h->combos : nullptr);
  {
    const double w = h->L * (1.0 + h->s + h->s + (combos ? h->ncombo : 0));
    ProfScope ps(h, P_STAGE, 8.0 * w, h->L * 2.0 * h->s * (h->s + (combos ? h->ncombo : 0)));
    launch_stage_states(h->g, sa, h->st);
  }
  if (combos && h->coef) {
    const int ncf = combo_coef_fields(h->g.op);
    ProfScope ps(h, P_STAGE, 8.0 * h->npts * (2.0 + ncf) * h->coef_list.n,
                 (ncf == 16 ? 52.0 : 10.0) * h->npts * h->coef_list.n);
    launch_combo_coef(h->g, h->combos, h->coef_list, dt, h->coef, h->st);
  }
  ResidualArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.s = h->s;
  // the kernel forms rhs_k = -sum_i Q[i][k] F_i; Q = (T^{-1})^T gives -(T^{-1} (x) I) F
  for (int i = 0; i < h->s; ++i)
    for (int k = 0; k < h->s; ++k) ra.Q[i * h->s + k] = h->tab.Tinv[k * h->s + i];
  for (int i = 0; i < h->s; ++i) ra.tstage[i] = t_n + h->tab.c[i] * dt;
  ra.forcing = h->cfg.forcing;
  ra.Y = h->Y;
  ra.K = K;
  ra.rhs = rhs;
  ra.Fraw = Fraw;
  ra.partials = h->partials;
  const int nb = residual_blocks(h->g);
  {
    const double w = h->L * (2.0 * h->s + (rhs ? h->s : 0) + (Fraw ? h->s : 0));
    ProfScope ps(h, P_RESID, 8.0 * w,
                 h->npts * h->s * (n_flops_per_point(h->g.op) + 4.0 * h->C + (rhs ? 2.0 * h->s * h->C : 0)));
    launch_residual(h->g, ra, h->st);
  }
  {
    ProfScope ps(h, P_REDUCE, 8.0 * nb, nb);
    launch_reduce(h->partials, nb, 1, 1, h->dscal + 201, h->st);
  }
}

// ||F(k = 0)||^2 into dscal[201], the reference of the Newton tolerance.  With
// k = 0 every stage reads Y_i = u_n, so for an autonomous N the s stage
// residuals are all -N(u_n) (and -G(u_n) on the DAE constraint rows): one stage
// is evaluated and f0_scale(h) = s multiplies its square norm.  A time-
// dependent source takes the full evaluation (scale 1).
double f0_scale(const irk_handle* h) { return h->cfg.forcing ? 1.0 : (double)h->s; }

void launch_f0_norm(irk_handle* h, double t_n, double dt) {
  if (h->cfg.forcing) {
    cudaMemsetAsync(h->yhat, 0, sizeof(double) * h->s * h->L, h->st);
    launch_eval_residual(h, t_n, dt, h->yhat, h->rhs, nullptr, false);
    return;
  }
  cudaMemsetAsync(h->yhat, 0, sizeof(double) * h->L, h->st);
  ResidualArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.s = 1;
  ra.Q[0] = 1.0;
  ra.tstage[0] = t_n;
  ra.Y = h->u;
  ra.K = h->yhat;
  ra.partials = h->partials;
  const int nb = residual_blocks(h->g);
  {
    ProfScope ps(h, P_RESID, 16.0 * h->L, h->npts * (n_flops_per_point(h->g.op) + 4.0 * h->C));
    launch_residual(h->g, ra, h->st);
  }
  {
    ProfScope ps(h, P_REDUCE, 8.0 * nb, nb);
    launch_reduce(h->partials, nb, 1, 1, h->dscal + 201, h->st);
  }
}

irk_status eval_residual(irk_handle* h, double t_n, double dt, const double* K, double* rhs,
                         double* Fraw, bool combos, double* fnorm) {
  launch_eval_residual(h, t_n, dt, K, rhs, Fraw, combos);
  // the norm, plus (slots 320..) the device-FGMRES iteration counters
  TRY(sync_read(h, h->dscal + 201, 140));
  *fnorm = std::sqrt(h->hbuf[0]);
  return IRK_OK;
}

// Device-FGMRES counters: dscal[320 + 2 blk] = iterations so far (all cycles),
// dscal[321 + 2 blk] = non-finite flag.  hbuf holds dscal[201..340] after a
// residual evaluation.
irk_status collect_fg_counters(irk_handle* h) {
  for (int blk = 0; blk < h->tab.nblk; ++blk) {
    const double its = h->hbuf[320 - 201 + 2 * blk];
    const double bad = h->hbuf[321 - 201 + 2 * blk];
    const long long d = (long long)(its - h->fg_seen_its[blk]);
    if (d > 0) {
      h->stats.krylov_its += (int)d;
      h->stats.prec_apps += (int)d * h->tab.bsize[blk];
      h->stats.vcycles += (int)d * h->fg_body_vcycles[blk];
      h->stats.poisson_vcycles += (int)d * h->fg_body_pvcycles[blk];
      h->stats.kernel_launches += d * h->fg_body_launches[blk];
    }
    h->fg_seen_its[blk] = its;
    if (bad != 0.0) {
      h->err = "non-finite Krylov vector";
      return IRK_ERR_KRYLOV_BREAKDOWN;
    }
  }
  return IRK_OK;
}

void drop_fg_graphs(irk_handle* h) {
  for (int k = 0; k < IRK_MAXS; ++k)
    if (h->fgexec[k]) {
      cudaGraphExecDestroy(h->fgexec[k]);
      h->fgexec[k] = nullptr;
    }
}

// One restart cycle of FGMRES on block blk, captured into the graph that
// stream `outer` is capturing:
//   prefix  z = rhs_blk - U dk_hat (Eq. D+U), x = 0, beta = ||z||, V_0 = z/beta
//   WHILE   z_j = L_P v_j; w = D z_j (Z_j = z_j); fused CGS2 + Arnoldi/Givens step
//   suffix  y = R^{-1} g; x += Z y
// The loop body is captured on stream `inner`.  The loop ends on the device
// (Arnoldi step of k_fg_gs2) after at most m iterations.
struct CapCounts {
  long long fixed = 0, body = 0;
  int vcycles = 0, pvcycles = 0;
};

cudaError_t capture_block_solve(irk_handle* h, double dt, int blk, cudaStream_t outer,
                                cudaStream_t inner, CapCounts* cc) {
  const int a0 = h->tab.bstart[blk], bs = h->tab.bsize[blk];
  const long long Lb = (long long)bs * h->L;
  const long long ldv = Lb;
  FGState* fs = h->fgs + blk;
  double* x = h->yhat + (long long)a0 * h->L;
  const double* b = h->rhs + (long long)a0 * h->L;
  cudaStream_t saved_st = h->st;
  h->st = outer;
  const long long l_start = h->stats.kernel_launches;
  // the conditional handle lives in the graph being captured on `outer`
  cudaStreamCaptureStatus cst;
  cudaGraph_t G = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(outer, &cst, nullptr, &G, nullptr, nullptr, nullptr);
  // (an invalidated capture has no usable graph or dependency list)
  if (e == cudaSuccess && cst != cudaStreamCaptureStatusActive) e = cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle cond = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, G, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) { h->st = saved_st; return e; }
  // ---- prefix
  if (blk < h->tab.nblk - 1) {
    upper_coupling(h, dt, blk, h->zbuf);
    b = h->zbuf;
  }
  cudaMemsetAsync(x, 0, sizeof(double) * Lb, outer);
  {
    ProfScope ps(h, P_NORM, 8.0 * Lb, 2.0 * Lb);
    launch_norm2(b, Lb, h->partials, outer);
  }
  {
    ProfScope ps(h, P_REDUCE, 0, 0);
    launch_reduce(h->partials, blas_blocks(Lb), 1, 1, h->dscal + 310, outer);
  }
  {
    ProfScope ps(h, P_SCALE, 0, 0);
    launch_fg_init(fs, h->dscal + 310, h->dscal + 300, cond, outer);
  }
  {
    ProfScope ps(h, P_SCALE, 16.0 * Lb, (double)Lb);
    launch_fg_scale(b, fs, h->V, ldv, h->prec_in, Lb, outer);
  }
  // ---- WHILE node after the prefix
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  e = cudaStreamGetCaptureInfo(outer, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
  if (e == cudaSuccess && cst != cudaStreamCaptureStatusActive) e = cudaErrorStreamCaptureInvalidated;
  cudaGraphNode_t wnode = nullptr;
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, G, deps, nullptr, ndeps, &np);
    if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
  }
  cc->fixed += h->stats.kernel_launches - l_start;
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(inner, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    h->st = inner;
    const long long l0 = h->stats.kernel_launches;
    const int v0 = h->stats.vcycles, pv0 = h->stats.poisson_vcycles;
    block_prec(h, dt, blk, h->prec_in, h->prec_out);
    {
      // w = D z_j with z_j = prec_out; Z_j = z_j (j read on the device)
      const int s = h->s;
      StageOpArgs a;
      memset(&a, 0, sizeof(a));
      a.nrow = bs;
      a.dt = dt;
      for (int rr = 0; rr < bs; ++rr) {
        const int r = a0 + rr;
        OpRow& row = a.row[rr];
        row.y = h->w + (long long)rr * h->L;
        row.sigma = 1;
        for (int qq = 0; qq < bs; ++qq) {
          const int q = a0 + qq;
          OpTerm& t = row.t[row.nterm++];
          t.x = h->prec_out + (long long)qq * h->L;
          set_combo(h, t, r, q);
          t.m = h->tab.R[r * s + q];
          t.lin = (r == q) ? 1.0 : 0.0;
        }
      }
      a.copy_dst = h->Z;
      a.copy_src = h->prec_out;
      a.copy_len = Lb;
      a.copy_jdev = &fs->j;
      a.copy_ldv = ldv;
      run_stage_op(h, a);
    }
    double* dh1 = h->dscal;
    double* dh2 = h->dscal + 64;
    {
      ProfScope ps(h, P_FG_GS1, 0, 0);
      launch_fg_gs1(h->V, ldv, fs, h->w, Lb, h->partials, dh1, inner);
    }
    {
      ProfScope ps(h, P_FG_GS2, 0, 0);
      launch_fg_gs2(h->V, ldv, fs, dh1, h->w, Lb, h->partials, dh2, h->m, h->cfg.krylov_maxit,
                    h->dscal + 320 + 2 * blk, cond, inner);
    }
    {
      ProfScope ps(h, P_FG_NEXT, 0, 0);
      launch_fg_next(h->V, ldv, fs, dh2, h->w, h->V, h->prec_in, Lb, h->m + 1, cond, inner);
    }
    cc->body = h->stats.kernel_launches - l0;
    cc->vcycles = h->stats.vcycles - v0;
    cc->pvcycles = h->stats.poisson_vcycles - pv0;
    h->st = outer;
    cudaGraph_t bout = nullptr;
    e = cudaStreamEndCapture(inner, &bout);
  }
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(outer, &wnode, nullptr, 1,
                                            cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) {
    const long long l1 = h->stats.kernel_launches;
    {
      ProfScope ps(h, P_LINCOMB, 0, 0);
      launch_fg_solve(fs, outer);
    }
    {
      ProfScope ps(h, P_LINCOMB, 0, 0);
      launch_fg_lincomb(x, h->Z, ldv, fs, Lb, outer);
    }
    cc->fixed += h->stats.kernel_launches - l1;
  }
  h->st = saved_st;
  return e;
}

// The block solve of the captured path launched kernel by kernel (per-kernel
// timing, cfg.profile = 1): the same prefix, body and suffix kernels as
// capture_block_solve, with a zero conditional handle; the host reads the
// FGState's loop flag after each body.  j = body index, so the algorithmic
// bytes and flops of the CGS2 kernels are known here.
irk_status direct_block_solve(irk_handle* h, double dt, int blk) {
  const int a0 = h->tab.bstart[blk], bs = h->tab.bsize[blk], s = h->s;
  const long long Lb = (long long)bs * h->L, ldv = Lb;
  FGState* fs = h->fgs + blk;
  double* x = h->yhat + (long long)a0 * h->L;
  const double* b = h->rhs + (long long)a0 * h->L;
  if (blk < h->tab.nblk - 1) {
    upper_coupling(h, dt, blk, h->zbuf);
    b = h->zbuf;
  }
  CK(cudaMemsetAsync(x, 0, sizeof(double) * Lb, h->st));
  {
    ProfScope ps(h, P_NORM, 8.0 * Lb, 2.0 * Lb);
    launch_norm2(b, Lb, h->partials, h->st);
  }
  {
    ProfScope ps(h, P_REDUCE, 8.0 * blas_blocks(Lb), blas_blocks(Lb));
    launch_reduce(h->partials, blas_blocks(Lb), 1, 1, h->dscal + 310, h->st);
  }
  {
    ProfScope ps(h, P_FG_CTL, 0, 0);
    launch_fg_init(fs, h->dscal + 310, h->dscal + 300, 0, h->st);
  }
  {
    ProfScope ps(h, P_SCALE, 16.0 * Lb, (double)Lb);
    launch_fg_scale(b, fs, h->V, ldv, h->prec_in, Lb, h->st);
  }
  for (int j = 0; j <= h->m; ++j) {
    int stopped = 1;
    CK(cudaMemcpyAsync(&stopped, &fs->stopped, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    prof_harvest(h);
    if (stopped) break;
    block_prec(h, dt, blk, h->prec_in, h->prec_out);
    StageOpArgs a;
    memset(&a, 0, sizeof(a));
    a.nrow = bs;
    a.dt = dt;
    for (int rr = 0; rr < bs; ++rr) {
      const int r = a0 + rr;
      OpRow& row = a.row[rr];
      row.y = h->w + (long long)rr * h->L;
      row.sigma = 1;
      for (int qq = 0; qq < bs; ++qq) {
        const int q = a0 + qq;
        OpTerm& t = row.t[row.nterm++];
        t.x = h->prec_out + (long long)qq * h->L;
        set_combo(h, t, r, q);
        t.m = h->tab.R[r * s + q];
        t.lin = (r == q) ? 1.0 : 0.0;
      }
    }
    a.copy_dst = h->Z;
    a.copy_src = h->prec_out;
    a.copy_len = Lb;
    a.copy_jdev = &fs->j;
    a.copy_ldv = ldv;
    run_stage_op(h, a);
    const double nv = j + 1;
    double* dh1 = h->dscal;
    double* dh2 = h->dscal + 64;
    {
      // V_0..V_j and w in; one FMA per value and basis vector
      ProfScope ps(h, P_FG_GS1, 8.0 * Lb * (nv + 1), 2.0 * Lb * nv);
      launch_fg_gs1(h->V, ldv, fs, h->w, Lb, h->partials, dh1, h->st);
    }
    {
      // w -= V h1 (nv FMAs), then V^T w and ||w||^2 (nv + 1 FMAs): w in and out
      ProfScope ps(h, P_FG_GS2, 8.0 * Lb * (nv + 2), 2.0 * Lb * (2.0 * nv + 1.0));
      launch_fg_gs2(h->V, ldv, fs, dh1, h->w, Lb, h->partials, dh2, h->m, h->cfg.krylov_maxit,
                    h->dscal + 320 + 2 * blk, 0, h->st);
    }
    {
      // V_{j+1} = (w - V h2) / h: V and w in, V_{j+1} and the preconditioner input out
      ProfScope ps(h, P_FG_NEXT, 8.0 * Lb * (nv + 3), 2.0 * Lb * nv + Lb);
      launch_fg_next(h->V, ldv, fs, dh2, h->w, h->V, h->prec_in, Lb, h->m + 1, 0, h->st);
    }
  }
  {
    ProfScope ps(h, P_FG_CTL, 0, 0);
    launch_fg_solve(fs, h->st);
  }
  {
    // k basis vectors of Z and x in, x out (k <= m; the count is on the device)
    ProfScope ps(h, P_LINCOMB, 0, 0);
    launch_fg_lincomb(x, h->Z, ldv, fs, Lb, h->st);
  }
  return IRK_OK;
}

// Standalone graph of one block solve (used when the whole-step graph is not).
irk_status build_fg_graph(irk_handle* h, double dt, int blk) {
  const irk_stats saved = h->stats;
  cudaGraph_t G = nullptr;
  CK(cudaGraphCreate(&G, 0));
  cudaError_t e = cudaStreamBeginCaptureToGraph(h->st, G, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal);
  CapCounts cc;
  if (e == cudaSuccess) {
    e = capture_block_solve(h, dt, blk, h->st, h->st_aux, &cc);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->st, &out);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->fgexec[blk], G, 0);
  cudaGraphDestroy(G);
  h->fg_fixed_launches[blk] = cc.fixed;
  h->fg_body_launches[blk] = cc.body;
  h->fg_body_vcycles[blk] = cc.vcycles;
  h->fg_body_pvcycles[blk] = cc.pvcycles;
  h->stats = saved;
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->fgexec[blk] = nullptr;
    return IRK_ERR_CUDA;
  }
  return IRK_OK;
}

// ---------------------------------------------------------------------------
// Whole IRK step as one CUDA graph (Algorithm 1 with the Newton loop on the
// device):
//   k = 0; F, ||F(0)||; k_newton_first
//   WHILE (Newton): MG setup; block solves (each with its own FGMRES WHILE);
//                   k += (Q0 R0 (x) I) dk_hat; F; k_newton_ctl
//   u_{n+1} = u_n + dt sum b_i k_i
// k_newton_ctl applies the host loop's tests (tolerance, iteration limit,
// growth, non-finite residual) and the same inexact-Newton forcing term; the
// host reads one status block after the graph.  Not used with a time-
// dependent source (its stage times would be baked into the graph).
// Newton starting value of a collocation method (initial_guess = 2): the
// previous step's stages are the derivative of its collocation polynomial at
// t_{n-1} + c_i h_old, so k_j = sum_i k_i l_i(1 + c_j h/h_old) (l_i the
// Lagrange basis on the abscissae) extrapolates it to this step's nodes.
constexpr int kExtrapSlot = 450;  // dscal[450 .. 450 + s*s)

bool use_extrapolation(const irk_handle* h) {
  return h->cfg.initial_guess == 2 && h->tab.collocation && h->s > 1;
}

// Upload E for this step's ratio h/h_old (identity when there is no previous
// step); the captured graphs read it from device memory.
irk_status prepare_guess(irk_handle* h, double dt) {
  if (!use_extrapolation(h)) return IRK_OK;
  const double r = h->last_dt > 0 ? dt / h->last_dt : (h->last_dt < 0 ? 1.0 : 0.0);
  if (r == h->E_ratio) return IRK_OK;
  const int s = h->s;
  double* E = h->hbuf + 256;  // pinned; the previous upload has completed (steps synchronize)
  for (int j = 0; j < s; ++j)
    for (int i = 0; i < s; ++i) {
      if (r == 0.0) {
        E[j * s + i] = (i == j) ? 1.0 : 0.0;
        continue;
      }
      const long double th = 1.0L + (long double)h->tab.c[j] * r;
      long double l = 1.0L;
      for (int m = 0; m < s; ++m)
        if (m != i) l *= (th - h->tab.c[m]) / ((long double)h->tab.c[i] - h->tab.c[m]);
      E[j * s + i] = (double)l;
    }
  CK(cudaMemcpyAsync(h->dscal + kExtrapSlot, E, sizeof(double) * s * s, cudaMemcpyHostToDevice,
                     h->st));
  h->E_ratio = r;
  return IRK_OK;
}

irk_status build_step_graph(irk_handle* h, double dt) {
  if (h->stepexec) {
    cudaGraphExecDestroy(h->stepexec);
    h->stepexec = nullptr;
  }
  const irk_stats saved = h->stats;
  const int s = h->s;
  cudaGraph_t G = nullptr;
  CK(cudaGraphCreate(&G, 0));
  cudaGraphConditionalHandle ncond = 0;
  cudaError_t e = cudaGraphConditionalHandleCreate(&ncond, G, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(h->st, G, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  long long fixed = 0, newton_body = 0;
  CapCounts blkcc[IRK_MAXS];
  if (e == cudaSuccess) {
    const long long l0 = h->stats.kernel_launches;
    if (h->cfg.initial_guess >= 1) {
      // ||F(k=0)|| fixes the tolerance; Newton then starts from the previous
      // stages, extrapolated along the collocation polynomial (guess 2)
      launch_f0_norm(h, 0.0, dt);
      {
        ProfScope ps(h, P_SCALE, 0, 0);
        launch_newton_first(h->nws, h->dscal + 201, f0_scale(h), h->dscal + 300,
                            h->cfg.newton_rtol, h->cfg.krylov_rtol, ncond, h->st);
      }
      if (use_extrapolation(h)) {
        ProfScope ps(h, P_UPDATE, 16.0 * h->L * s, 2.0 * h->L * s * s);
        launch_stage_extrapolate(h->L, s, h->dscal + kExtrapSlot, h->K, h->st);
      }
      {
        ProfScope ps(h, P_SCALE, 0, 0);
        launch_zero_if_unforced(h->nws, h->K, (long long)s * h->L, h->st);
      }
      launch_eval_residual(h, 0.0, dt, h->K, h->rhs, nullptr, true);
      {
        ProfScope ps(h, P_SCALE, 0, 0);
        launch_newton_ctl(h->nws, h->dscal + 201, h->dscal + 300, h->cfg.newton_rtol,
                          h->cfg.newton_maxit, h->cfg.krylov_rtol, ncond, 0, h->st);
      }
    } else {
      cudaMemsetAsync(h->K, 0, sizeof(double) * s * h->L, h->st);
      launch_eval_residual(h, 0.0, dt, h->K, h->rhs, nullptr, true);
      {
        ProfScope ps(h, P_SCALE, 0, 0);
        launch_newton_first(h->nws, h->dscal + 201, 1.0, h->dscal + 300, h->cfg.newton_rtol,
                            h->cfg.krylov_rtol, ncond, h->st);
      }
    }
    fixed += h->stats.kernel_launches - l0;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(h->st, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e == cudaSuccess && cst != cudaStreamCaptureStatusActive) e = cudaErrorStreamCaptureInvalidated;
    cudaGraphNode_t wnode = nullptr;
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = ncond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&wnode, G, deps, nullptr, ndeps, &np);
      if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(h->st_aux, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaStream_t main = h->st;
      h->st = h->st_aux;
      const long long l1 = h->stats.kernel_launches;
      mg_setup(h, dt);
      for (int blk = h->tab.nblk - 1; blk >= 0 && e == cudaSuccess; --blk)
        e = capture_block_solve(h, dt, blk, h->st_aux, h->st_aux2, &blkcc[blk]);
      if (e == cudaSuccess) {
        {
          ProfScope ps(h, P_UPDATE, 8.0 * h->L * 3 * s, 2.0 * h->L * s * s);
          launch_stage_update(h->L, s, h->tab.TR, h->yhat, h->K, h->st);
        }
        if (h->g.op == IRK_OP_VSF_2D) {
          ProfScope ps(h, P_MEAN, 24.0 * h->npts * s, 2.0 * h->npts * s, 2);
          launch_remove_mean(h->npts, s, h->L, h->K + h->npts, h->partials, h->st);
        }
        launch_eval_residual(h, 0.0, dt, h->K, h->rhs, nullptr, true);
        {
          ProfScope ps(h, P_SCALE, 0, 0);
          launch_newton_ctl(h->nws, h->dscal + 201, h->dscal + 300, h->cfg.newton_rtol,
                            h->cfg.newton_maxit, h->cfg.krylov_rtol, ncond, 1, h->st);
        }
      }
      newton_body = h->stats.kernel_launches - l1;
      h->st = main;
      cudaGraph_t bout = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(h->st_aux, &bout);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(h->st, &wnode, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
      const long long l2 = h->stats.kernel_launches;
      ProfScope ps(h, P_UPDATE, 8.0 * h->L * (2 + s), 2.0 * h->L * s);
      launch_u_update(h->L, s, h->tab.b, dt, h->K, h->u, h->st);
      fixed += h->stats.kernel_launches - l2;
    }
    cudaGraph_t out = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(h->st, &out);
    if (e == cudaSuccess) e = e3;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->stepexec, G, 0);
  cudaGraphDestroy(G);
  h->stats = saved;
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->stepexec = nullptr;
    return IRK_ERR_CUDA;
  }
  // launches per Newton iteration outside the block loops, and per block
  long long blocks_fixed = 0;
  for (int blk = 0; blk < h->tab.nblk; ++blk) {
    blocks_fixed += blkcc[blk].fixed;
    h->fg_body_launches[blk] = blkcc[blk].body;
    h->fg_body_vcycles[blk] = blkcc[blk].vcycles;
    h->fg_body_pvcycles[blk] = blkcc[blk].pvcycles;
  }
  (void)blocks_fixed;
  h->step_fixed_launches = fixed;
  // launches of one Newton iteration without its Krylov-loop bodies (counted per iteration)
  h->step_newton_launches = newton_body;
  for (int blk = 0; blk < h->tab.nblk; ++blk) h->step_newton_launches -= blkcc[blk].body;
  h->step_dt = dt;
  return IRK_OK;
}

// One IRK step through the step graph.  Returns IRK_OK, a Newton/Krylov
// status, or IRK_ERR_INVALID when the graph cannot be used (caller falls back).
irk_status graph_step(irk_handle* h, double dt) {
  if (!h->cfg.use_graphs || h->cfg.profile || h->cfg.forcing || h->step_failed || !h->st_aux ||
      !h->st_aux2 || h->cfg.nonlinear_variant == 4 || h->cfg.dae_solver == 1)
    return IRK_ERR_INVALID;
  TraceRange tr("step_graph");
  if (!h->stepexec || h->step_dt != dt) {
    if (build_step_graph(h, dt) != IRK_OK) {
      h->step_failed = true;
      return IRK_ERR_INVALID;
    }
  }
  CK(cudaGraphLaunch(h->stepexec, h->st));
  // Newton status (dscal[400..406]) and Krylov counters (dscal[320..330])
  CK(cudaMemcpyAsync(h->hbuf, h->dscal + 300, sizeof(double) * 110, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const double* nw = h->hbuf + 100;  // dscal[400..]
  if ((int)nw[5] == kGuessRejected) {
    // the warm start was worse than zero stages: run the step again from
    // zero, from the saved state (the graph's final update has run)
    h->stats.kernel_launches += h->step_fixed_launches;
    CK(cudaMemcpyAsync(h->u, h->u_save, sizeof(double) * h->L, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemsetAsync(h->K, 0, sizeof(double) * h->s * h->L, h->st));
    CK(cudaGraphLaunch(h->stepexec, h->st));
    CK(cudaMemcpyAsync(h->hbuf, h->dscal + 300, sizeof(double) * 110, cudaMemcpyDeviceToHost,
                       h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  const int its = (int)nw[4];
  // zero stages cannot be rejected again (ratio 1); if they were, report divergence
  const int status = ((int)nw[5] == kGuessRejected) ? (int)IRK_ERR_NEWTON_DIVERGED : (int)nw[5];
  h->stats.newton_its += its;
  h->stats.max_newton_its = std::max(h->stats.max_newton_its, its);
  h->stats.final_rel_res = nw[2];
  h->stats.kernel_launches += h->step_fixed_launches + (long long)its * h->step_newton_launches;
  for (int blk = 0; blk < h->tab.nblk; ++blk) {
    const double kits = h->hbuf[20 + 2 * blk];  // dscal[320 + 2 blk]
    const double bad = h->hbuf[21 + 2 * blk];
    const long long d = (long long)(kits - h->fg_seen_its[blk]);
    if (d > 0) {
      h->stats.krylov_its += (int)d;
      h->stats.prec_apps += (int)d * h->tab.bsize[blk];
      h->stats.vcycles += (int)d * h->fg_body_vcycles[blk];
      h->stats.poisson_vcycles += (int)d * h->fg_body_pvcycles[blk];
      h->stats.kernel_launches += d * h->fg_body_launches[blk];
    }
    h->fg_seen_its[blk] = kits;
    if (bad != 0.0) { h->err = "non-finite Krylov vector"; return IRK_ERR_KRYLOV_BREAKDOWN; }
  }
  if (status == 0) return IRK_OK;
  char buf[160];
  if (status == IRK_ERR_NEWTON_MAXIT) {
    snprintf(buf, sizeof buf, "Newton did not reach rtol %.1e in %d iterations (rel %.3e)",
             h->cfg.newton_rtol, its, nw[2]);
  } else {
    snprintf(buf, sizeof buf, "Newton diverged (rel %.3e after %d iterations)", nw[2], its);
  }
  h->err = buf;
  return (irk_status)status;
}

// All block solves of one Newton iteration through the device-resident graphs.
// Returns false (and leaves no work queued) when graphs cannot be used.
bool fg_device_solve(irk_handle* h, double dt, double eta) {
  if (!h->cfg.use_graphs || h->cfg.profile || h->fg_failed || !h->st_aux) return false;
  if (h->fg_dt != dt) {
    drop_fg_graphs(h);
    h->fg_dt = dt;
  }
  for (int blk = 0; blk < h->tab.nblk; ++blk)
    if (!h->fgexec[blk] && build_fg_graph(h, dt, blk) != IRK_OK) {
      drop_fg_graphs(h);
      h->fg_failed = true;
      return false;
    }
  h->hbuf[400] = eta;
  if (cudaMemcpyAsync(h->dscal + 300, h->hbuf + 400, sizeof(double), cudaMemcpyHostToDevice,
                      h->st) != cudaSuccess)
    return false;
  for (int blk = h->tab.nblk - 1; blk >= 0; --blk) {
    cudaGraphLaunch(h->fgexec[blk], h->st);
    h->stats.kernel_launches += h->fg_fixed_launches[blk];
  }
  return true;
}

// Block backward substitution of Algorithm 1 on h->rhs into h->yhat: the
// device-resident FGMRES graphs when available, else the host-driven loop.
// ---------------------------------------------------------------------------
// Block forward solve of Eq. vsf-system-2 (VSF, dae_solver = 1).  With the
// Picard linearization the advection acts on omega with the lagged stream
// function only, so once one Schur block's unknowns are ordered (omega rows,
// psi rows) its system is block lower triangular: the omega rows alone are
// the eta/gamma* block system of Sec. 4 (solved by FGMRES with the omega
// part of L_P to rtol), and each psi row is then the Poisson problem
// dt (x_omega + L x_psi) = z_psi, i.e. (-L) x_psi = x_omega - z_psi / dt,
// solved by FGMRES with the Poisson V-cycle to rtol.  Omega vectors of a
// block are stored row after row, npts values each.

// y = D x on the omega rows of block blk (Picard: no J_A(x_psi, wbar) term)
void omega_block_matvec(irk_handle* h, double dt, int blk, const double* x, double* y,
                        const double* copy_src, double* copy_dst) {
  const int a0 = h->tab.bstart[blk], bs = h->tab.bsize[blk], s = h->s;
  StageOpArgs a;
  memset(&a, 0, sizeof(a));
  a.nrow = bs;
  a.dt = dt;
  a.vsf_omega_only = 1;
  for (int rr = 0; rr < bs; ++rr) {
    const int r = a0 + rr;
    OpRow& row = a.row[rr];
    row.y = y + (long long)rr * h->npts;
    row.sigma = 1;
    for (int qq = 0; qq < bs; ++qq) {
      const int q = a0 + qq;
      OpTerm& t = row.t[row.nterm++];
      t.x = x + (long long)qq * h->npts;
      set_combo(h, t, r, q);
      t.m = h->tab.R[r * s + q];
      t.lin = (r == q) ? 1.0 : 0.0;
    }
  }
  a.copy_dst = copy_dst;
  a.copy_src = copy_src;
  a.copy_len = copy_dst ? (long long)bs * h->npts : 0;
  run_stage_op(h, a);
}

// omega rows of z_blk = rhs_blk - sum_{l beyond blk} U_{r,l} yhat_l (the psi
// rows of U vanish: M = diag(I, 0) and no linear term off the diagonal)
void omega_upper_coupling(irk_handle* h, double dt, int blk, double* z) {
  const int a0 = h->tab.bstart[blk], bs = h->tab.bsize[blk], s = h->s;
  StageOpArgs a;
  memset(&a, 0, sizeof(a));
  a.nrow = bs;
  a.dt = dt;
  a.vsf_omega_only = 1;
  for (int rr = 0; rr < bs; ++rr) {
    const int r = a0 + rr;
    OpRow& row = a.row[rr];
    row.y = z + (long long)rr * h->npts;
    row.base = h->rhs + (long long)r * h->L;
    row.alpha = 1;
    row.sigma = -1;
    for (int l = a0 + bs; l < s; ++l) {
      OpTerm& t = row.t[row.nterm++];
      t.x = h->yhat + (long long)l * h->L;
      set_combo(h, t, r, l);
      t.m = h->tab.R[r * s + l];
      t.lin = 0;
    }
  }
  run_stage_op(h, a);
}

// z = the omega part of L_P (Eq. Lprec) for block blk
void omega_block_prec(irk_handle* h, double dt, int blk, const double* v, double* z) {
  const int a = h->tab.bstart[blk], bs = h->tab.bsize[blk], s = h->s;
  const double eta = h->tab.eta[blk];
  const double cdiff = dt * h->g.nu;
  vcycle(h, a, MG_ADVECTIVE, 1, eta, dt, cdiff, 0, v, z);
  if (bs == 1) return;
  const int b = a + 1;
  const double gamma = (h->cfg.gamma_mode == 1) ? eta : h->tab.gamma_star[blk];
  // r_b' = v_b - (coupling row (b, a)) z_a
  StageOpArgs op;
  memset(&op, 0, sizeof(op));
  op.nrow = 1;
  op.dt = dt;
  op.vsf_omega_only = 1;
  OpRow& row = op.row[0];
  row.y = h->tmp;
  row.base = v + h->npts;
  row.alpha = 1;
  row.sigma = -1;
  row.nterm = 1;
  row.t[0].x = z;
  set_combo(h, row.t[0], b, a);
  row.t[0].m = h->tab.R[b * s + a];
  row.t[0].lin = 0;
  run_stage_op(h, op);
  vcycle(h, b, MG_ADVECTIVE, 1, gamma, dt, cdiff, 0, h->tmp, z + h->npts);
}

// x = (-L)^+ b by FGMRES with the Poisson V-cycle (b's mean removed first)
irk_status poisson_fgmres(irk_handle* h, double* b, double* x, double rtol) {
  const long long n = h->npts;
  {
    ProfScope ps(h, P_MEAN, 24.0 * n, 2.0 * n, 2);
    launch_remove_mean(h->npts, 1, n, b, h->partials, h->st);
  }
  auto step = [&](int j) -> irk_status {
    vcycle(h, -1, MG_DIFFUSION, 1, 0.0, 0.0, 1.0, 1, h->prec_in, h->prec_out);
    {
      ProfScope ps(h, P_POISSON, 16.0 * n, 6.0 * n);
      launch_neg_laplacian(h->g, h->prec_out, h->w, h->st);
    }
    CK(cudaMemcpyAsync(h->Z + (long long)j * n, h->prec_out, sizeof(double) * n,
                       cudaMemcpyDeviceToDevice, h->st));
    return IRK_OK;
  };
  auto apply = [&](const double* xin, double* y) {
    ProfScope ps(h, P_POISSON, 16.0 * n, 6.0 * n);
    launch_neg_laplacian(h->g, xin, y, h->st);
  };
  auto counted = [&]() {};
  int its = 0;
  double rr = 0;
  return fgmres_core(h, n, h->m, h->cfg.krylov_maxit, h->V, h->Z, h->w, h->prec_in, b, x, rtol,
                     &its, &rr, step, apply, counted);
}

irk_status vsf_forward_solve(irk_handle* h, double dt, double rtol) {
  TraceRange tr("vsf_forward_solve");
  const long long n = h->npts;
  for (int blk = h->tab.nblk - 1; blk >= 0; --blk) {
    const int a0 = h->tab.bstart[blk], bs = h->tab.bsize[blk];
    // omega right-hand side and solution, row after row, in zbuf
    double* zw = h->zbuf;
    double* xw = h->zbuf + (long long)bs * n;
    if (blk < h->tab.nblk - 1) {
      omega_upper_coupling(h, dt, blk, zw);
    } else {
      for (int rr = 0; rr < bs; ++rr)
        CK(cudaMemcpyAsync(zw + rr * n, h->rhs + (long long)(a0 + rr) * h->L, sizeof(double) * n,
                           cudaMemcpyDeviceToDevice, h->st));
    }
    const long long Lb = (long long)bs * n;
    auto step = [&](int j) -> irk_status {
      omega_block_prec(h, dt, blk, h->prec_in, h->prec_out);
      omega_block_matvec(h, dt, blk, h->prec_out, h->w, h->prec_out, h->Z + (long long)j * Lb);
      return IRK_OK;
    };
    auto apply = [&](const double* xin, double* y) {
      omega_block_matvec(h, dt, blk, xin, y, nullptr, nullptr);
    };
    auto counted = [&]() {
      h->stats.krylov_its += 1;
      h->stats.prec_apps += bs;
    };
    int its = 0;
    double rr = 0;
    TRY(fgmres_core(h, Lb, h->m, h->cfg.krylov_maxit, h->V, h->Z, h->w, h->prec_in, zw, xw, rtol,
                    &its, &rr, step, apply, counted));
    for (int q = 0; q < bs; ++q) {
      double* yrow = h->yhat + (long long)(a0 + q) * h->L;
      CK(cudaMemcpyAsync(yrow, xw + q * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
      // Poisson right-hand side x_omega - z_psi / dt
      {
        ProfScope ps(h, P_AXPBY, 40.0 * n, 3.0 * n, 2);
        launch_axpby(h->tmp2, 1.0, xw + q * n, 0.0, n, h->st);
        launch_axpby(h->tmp2, -1.0 / dt, h->rhs + (long long)(a0 + q) * h->L + n, 1.0, n, h->st);
      }
      TRY(poisson_fgmres(h, h->tmp2, yrow + n, rtol));
    }
  }
  return IRK_OK;
}

irk_status solve_blocks(irk_handle* h, double dt, double rtol, bool* on_device) {
  TraceRange tr("block_solves");
  if (h->cfg.dae_solver == 1) {
    *on_device = false;
    return vsf_forward_solve(h, dt, rtol);
  }
  *on_device = fg_device_solve(h, dt, rtol);
  if (*on_device) return IRK_OK;
  if (h->cfg.profile && h->cfg.use_graphs && !h->fg_failed) {
    // per-kernel timing of the path the graphs run: their kernels, one launch each
    h->hbuf[400] = rtol;
    CK(cudaMemcpyAsync(h->dscal + 300, h->hbuf + 400, sizeof(double), cudaMemcpyHostToDevice,
                       h->st));
    for (int blk = h->tab.nblk - 1; blk >= 0; --blk) TRY(direct_block_solve(h, dt, blk));
    *on_device = true;
    return IRK_OK;
  }
  for (int blk = h->tab.nblk - 1; blk >= 0; --blk) {
    const int a0 = h->tab.bstart[blk];
    const double* z = h->rhs + (long long)a0 * h->L;
    if (blk < h->tab.nblk - 1) {
      upper_coupling(h, dt, blk, h->zbuf);
      z = h->zbuf;
    }
    int its = 0;
    double rr = 0;
    TRY(fgmres(h, dt, blk, z, h->yhat + (long long)a0 * h->L, rtol, &its, &rr));
  }
  return IRK_OK;
}

// out = J v for the true stage Jacobian (Eq. keq4 before any approximation):
// (J v)_i = M v_i - dt J(Y_i) sum_j a_ij v_j at the stage states in h->Y.
void full_jvp(irk_handle* h, double dt, const double* v, double* out, double* wscratch) {
  const int s = h->s;
  StageStateArgs wa;
  set_stage_args(h, wa, 1.0, nullptr, v, wscratch, nullptr);
  {
    ProfScope ps(h, P_STAGE, 8.0 * h->L * 2 * s, 2.0 * h->L * s * s);
    launch_stage_states(h->g, wa, h->st);
  }
  for (int i = 0; i < s; i += 2) {
    StageOpArgs a;
    memset(&a, 0, sizeof(a));
    a.nrow = std::min(2, s - i);
    a.dt = dt;
    for (int rr = 0; rr < a.nrow; ++rr) {
      const long long off = (long long)(i + rr) * h->L;
      OpRow& row = a.row[rr];
      row.y = out + off;
      row.sigma = 1;
      row.nterm = 2;
      row.t[0].x = v + off;
      row.t[0].combo = nullptr;
      row.t[0].m = 1.0;
      row.t[0].lin = 0.0;
      row.t[1].x = wscratch + off;
      row.t[1].combo = h->Y + off;
      row.t[1].m = 0.0;
      row.t[1].lin = 1.0;
    }
    run_stage_op(h, a);
  }
}

// z = P^{-1} r for P the variant-3 approximation of the stage Jacobian:
// P^{-1} = (T R (x) I) B^{-1} (T^{-1} (x) I), B the block upper triangular
// matrix of Algorithm 1, applied by one block backward substitution with
// inner FGMRES solves to relative tolerance rtol.
irk_status alg1_sweep(irk_handle* h, double dt, const double* r, double* z, double rtol) {
  const int s = h->s;
  const long long Lo = (long long)s * h->L;
  {
    ProfScope ps(h, P_UPDATE, 8.0 * Lo * 2, 2.0 * h->L * s * s);
    CK(cudaMemsetAsync(h->rhs, 0, sizeof(double) * Lo, h->st));
    launch_stage_update(h->L, s, h->tab.Tinv, r, h->rhs, h->st);
  }
  bool on_device = false;
  TRY(solve_blocks(h, dt, rtol, &on_device));
  {
    ProfScope ps(h, P_UPDATE, 8.0 * Lo * 2, 2.0 * h->L * s * s);
    CK(cudaMemsetAsync(z, 0, sizeof(double) * Lo, h->st));
    launch_stage_update(h->L, s, h->tab.TR, h->yhat, z, h->st);
  }
  if (h->g.op == IRK_OP_VSF_2D) {
    // constant psi is in the null space of J; keep the iterates free of it
    ProfScope ps(h, P_MEAN, 24.0 * h->npts * s, 2.0 * h->npts * s, 2);
    launch_remove_mean(h->npts, s, h->L, z + h->npts, h->partials, h->st);
  }
  if (on_device) {
    TRY(sync_read(h, h->dscal + 201, 140));
    TRY(collect_fg_counters(h));
  }
  return IRK_OK;
}

// Exact Newton update (variant 4): solve J x = F (F in h->fo) by FGMRES over
// all stages, right-preconditioned by one Algorithm-1 sweep, then K -= x.
irk_status exact_newton_update(irk_handle* h, double dt, double rtol) {
  TraceRange tr("exact_newton_update");
  const long long Lo = (long long)h->s * h->L;
  const double rtol_in = h->cfg.krylov_rtol;
  auto step = [&](int j) -> irk_status {
    double* zj = h->Zo + (long long)j * Lo;
    TRY(alg1_sweep(h, dt, h->Vo + (long long)j * Lo, zj, rtol_in));
    full_jvp(h, dt, zj, h->wo, h->jw);
    return IRK_OK;
  };
  auto apply = [&](const double* x, double* y) { full_jvp(h, dt, x, y, h->jw); };
  auto counted = [&]() { h->stats.outer_its += 1; };
  int its = 0;
  double rr = 0;
  TRY(fgmres_core(h, Lo, h->mo, h->cfg.krylov_maxit, h->Vo, h->Zo, h->wo, nullptr, h->fo, h->xo,
                  rtol, &its, &rr, step, apply, counted));
  ProfScope ps(h, P_AXPBY, 24.0 * Lo, 2.0 * Lo);
  launch_axpby(h->K, -1.0, h->xo, 1.0, Lo, h->st);
  return IRK_OK;
}

irk_status newton_step(irk_handle* h, double t_n, double dt) {
  TraceRange tr("newton");
  const int s = h->s;
  double f0 = 0, fn = 0, prev = 0, prev_rel = 0;
  if (h->cfg.initial_guess >= 1) {
    // ||F(k=0)|| fixes the tolerance; Newton then starts from the previous
    // stages, extrapolated along the collocation polynomial (guess 2)
    launch_f0_norm(h, t_n, dt);
    TRY(sync_read(h, h->dscal + 201, 1));
    f0 = std::sqrt(f0_scale(h) * h->hbuf[0]);
    if (use_extrapolation(h)) {
      ProfScope ps(h, P_UPDATE, 16.0 * h->L * s, 2.0 * h->L * s * s);
      launch_stage_extrapolate(h->L, s, h->dscal + kExtrapSlot, h->K, h->st);
    }
    if (f0 == 0.0) CK(cudaMemsetAsync(h->K, 0, sizeof(double) * s * h->L, h->st));
  } else {
    CK(cudaMemsetAsync(h->K, 0, sizeof(double) * s * h->L, h->st));
  }
  int it = 0;
  for (;; ++it) {
    TraceRange tri("newton_iteration");
    TRY(eval_residual(h, t_n, dt, h->K, h->rhs, h->fo, true, &fn));
    if (it == 0 && h->cfg.initial_guess >= 1 && f0 > 0 && fn > kGuessLimit * f0) {
      // the warm start is worse than zero stages: start from zero instead
      CK(cudaMemsetAsync(h->K, 0, sizeof(double) * s * h->L, h->st));
      TRY(eval_residual(h, t_n, dt, h->K, h->rhs, h->fo, true, &fn));
    }
    if (it > 0) TRY(collect_fg_counters(h));
    if (!std::isfinite(fn) || !std::isfinite(f0)) { h->err = "non-finite stage residual"; return IRK_ERR_NEWTON_DIVERGED; }
    if (it == 0 && h->cfg.initial_guess == 0) f0 = fn;
    const double rel = (f0 > 0) ? fn / f0 : 0.0;
    h->stats.final_rel_res = rel;
    if (f0 == 0 || rel <= h->cfg.newton_rtol) break;
    if (it >= h->cfg.newton_maxit) {
      char buf[160];
      snprintf(buf, sizeof buf, "Newton did not reach rtol %.1e in %d iterations (rel %.3e)",
               h->cfg.newton_rtol, it, rel);
      h->err = buf;
      return IRK_ERR_NEWTON_MAXIT;
    }
    if (it > 0 && rel > 1e3) { h->err = "Newton residual grew by 1e3"; return IRK_ERR_NEWTON_DIVERGED; }
    // inexact-Newton forcing term: tighten with the residual, finish in one
    // step once the observed quadratic rate allows it, never oversolve
    double eta_lin = std::min(h->cfg.krylov_rtol, rel);
    if (it > 0 && prev > 0 && fn > 0.5 * prev) eta_lin = std::min(eta_lin, 1e-3 * rel);
    if (it > 0 && prev_rel > 0 &&
        (rel / (prev_rel * prev_rel)) * rel * rel <= 0.25 * h->cfg.newton_rtol)
      eta_lin = std::min(eta_lin, 0.5 * h->cfg.newton_rtol / rel);
    eta_lin = std::max(eta_lin, 0.2 * h->cfg.newton_rtol / rel);
    eta_lin = std::max(eta_lin, 1e-13);
    prev = fn;
    prev_rel = rel;
    mg_setup(h, dt);
    if (h->cfg.nonlinear_variant == 4) {
      TRY(exact_newton_update(h, dt, eta_lin));
    } else {
      bool on_device = false;
      TRY(solve_blocks(h, dt, eta_lin, &on_device));
      ProfScope ps(h, P_UPDATE, 8.0 * h->L * 3 * s, 2.0 * h->L * s * s);
      launch_stage_update(h->L, s, h->tab.TR, h->yhat, h->K, h->st);
    }
    if (h->g.op == IRK_OP_VSF_2D) {
      ProfScope ps(h, P_MEAN, 24.0 * h->npts * s, 2.0 * h->npts * s, 2);
      launch_remove_mean(h->npts, s, h->L, h->K + h->npts, h->partials, h->st);
    }
    h->stats.newton_its += 1;
  }
  h->stats.max_newton_its = std::max(h->stats.max_newton_its, it);
  {
    ProfScope ps(h, P_UPDATE, 8.0 * h->L * (2 + s), 2.0 * h->L * s);
    launch_u_update(h->L, s, h->tab.b, dt, h->K, h->u, h->st);
  }
  return IRK_OK;
}

// One SDIRK step stage by stage: stage i is the single-stage problem
// M k_i = N(u_n + dt sum_{j<i} a_ij k_j + dt gamma k_i, t_n + c_i dt), solved
// by the stage solver (its own Newton loop, Algorithm 1 with one 1x1 block of
// shift 1/gamma) from the base state written into its u; then
// u_{n+1} = u_n + dt sum_i b_i k_i (Eq. update).
irk_status sdirk_sequential_step(irk_handle* h, double t_n, double dt) {
  irk_handle* in = h->inner;
  const int s = h->s;
  const size_t vb = sizeof(double) * h->L;
  for (int i = 0; i < s; ++i) {
    TraceRange tr("sdirk_stage");
    CK(cudaMemcpyAsync(in->u, h->u, vb, cudaMemcpyDeviceToDevice, h->st));
    if (i > 0) {
      ProfScope ps(h, P_UPDATE, 8.0 * h->L * (2 + i), 2.0 * h->L * i);
      launch_u_update(h->L, i, h->tab.A + i * s, dt, h->K, in->u, h->st);
    }
    // the stage solver restores its base from u_save if it restarts from zero
    CK(cudaMemcpyAsync(in->u_save, in->u, vb, cudaMemcpyDeviceToDevice, h->st));
    // Newton guess: this stage at the previous step (zero after a reset)
    if (h->cfg.initial_guess >= 1)
      CK(cudaMemcpyAsync(in->K, h->K + (long long)i * h->L, vb, cudaMemcpyDeviceToDevice, h->st));
    memset(&in->stats, 0, sizeof(in->stats));
    irk_status st = graph_step(in, dt);
    if (st == IRK_ERR_INVALID) st = newton_step(in, t_n + h->tab.c[i] * dt, dt);
    h->stats.newton_its += in->stats.newton_its;
    h->stats.max_newton_its = std::max(h->stats.max_newton_its, in->stats.max_newton_its);
    h->stats.krylov_its += in->stats.krylov_its;
    h->stats.prec_apps += in->stats.prec_apps;
    h->stats.vcycles += in->stats.vcycles;
    h->stats.poisson_vcycles += in->stats.poisson_vcycles;
    h->stats.outer_its += in->stats.outer_its;
    h->stats.kernel_launches += in->stats.kernel_launches;
    h->stats.final_rel_res = std::max(i == 0 ? 0.0 : h->stats.final_rel_res, in->stats.final_rel_res);
    if (st != IRK_OK) {
      h->err = "SDIRK stage " + std::to_string(i) + ": " + in->err;
      cudaMemsetAsync(in->K, 0, vb, h->st);
      return st;
    }
    CK(cudaMemcpyAsync(h->K + (long long)i * h->L, in->K, vb, cudaMemcpyDeviceToDevice, h->st));
  }
  ProfScope ps(h, P_UPDATE, 8.0 * h->L * (2 + s), 2.0 * h->L * s);
  launch_u_update(h->L, s, h->tab.b, dt, h->K, h->u, h->st);
  return IRK_OK;
}

// ---------------------------------------------------------------------------
irk_status validate(const irk_config* c, std::string& err) {
  if (!c) { err = "null config"; return IRK_ERR_INVALID; }
  if (c->family < IRK_GAUSS || c->family > IRK_SDIRK) { err = "unknown family"; return IRK_ERR_INVALID; }
  if (c->family == IRK_SDIRK && !(c->stages == 1 || c->stages == 2 || c->stages == 3 || c->stages == 5)) { err = "SDIRK stages must be 1, 2, 3 or 5"; return IRK_ERR_INVALID; }
  if (c->family == IRK_SDIRK && c->stages > 1 && c->basis != IRK_BASIS_SCHUR) { err = "SDIRK has no eigenvector basis (one repeated eigenvalue): use the Schur basis"; return IRK_ERR_INVALID; }
  if (c->dirk_sequential != 0 && c->dirk_sequential != 1) { err = "dirk_sequential must be 0 or 1"; return IRK_ERR_INVALID; }
  if (c->dae_solver != 0 && c->dae_solver != 1) { err = "dae_solver must be 0 or 1"; return IRK_ERR_INVALID; }
  if (c->dae_solver == 1 && c->op != IRK_OP_VSF_2D) { err = "dae_solver 1 is defined for the VSF operator"; return IRK_ERR_INVALID; }
  if (c->dae_solver == 1 && c->nonlinear_variant == 4) { err = "dae_solver 1 solves the Picard system: nonlinear_variant 0..3"; return IRK_ERR_INVALID; }
  if (c->family == IRK_LOBATTO_IIIC && c->stages < 2) { err = "Lobatto IIIC needs stages >= 2"; return IRK_ERR_INVALID; }
  if (c->basis != IRK_BASIS_SCHUR && c->basis != IRK_BASIS_EIGEN) { err = "basis must be 0 (Schur) or 1 (eigenvectors)"; return IRK_ERR_INVALID; }
  if (c->stages < 1 || c->stages > IRK_MAXS) { err = "stages must be in 1..5"; return IRK_ERR_INVALID; }
  if (c->op < IRK_OP_DIFFUSION_1D || c->op > IRK_OP_VSF_2D) { err = "unknown op"; return IRK_ERR_INVALID; }
  const int want_mass = (c->op == IRK_OP_VSF_2D) ? IRK_MASS_DAE : IRK_MASS_IDENTITY;
  if (c->mass != want_mass) { err = "mass does not match op (DAE mass exactly for VSF)"; return IRK_ERR_INVALID; }
  if (c->n < 8 || c->n > 8192 || (c->n & (c->n - 1))) { err = "n must be a power of two in 8..8192"; return IRK_ERR_INVALID; }
  if (!(c->nu > 0) || !std::isfinite(c->nu)) { err = "nu must be positive"; return IRK_ERR_INVALID; }
  if (!(c->length > 0)) { err = "length must be positive"; return IRK_ERR_INVALID; }
  if (c->forcing != 0 && c->forcing != 1) { err = "forcing must be 0 or 1"; return IRK_ERR_INVALID; }
  if (c->forcing == 1 && !(c->op == IRK_OP_BURGERS_1D || c->op == IRK_OP_DIFFUSION_1D)) { err = "forcing 1 is defined for the 1D operators"; return IRK_ERR_INVALID; }
  if (c->forcing == 1 && c->length != 1.0) { err = "forcing 1 needs length 1"; return IRK_ERR_INVALID; }
  if (!(c->newton_rtol > 0) || c->newton_maxit < 1) { err = "bad Newton tolerance"; return IRK_ERR_INVALID; }
  if (!(c->krylov_rtol > 0) || c->krylov_restart < 1 || c->krylov_restart > 64 || c->krylov_maxit < 1) { err = "bad Krylov settings"; return IRK_ERR_INVALID; }
  if (c->nonlinear_variant < 0 || c->nonlinear_variant > 4) { err = "nonlinear_variant must be 0..4"; return IRK_ERR_INVALID; }
  if (c->gamma_mode != 0 && c->gamma_mode != 1) { err = "gamma_mode must be 0 or 1"; return IRK_ERR_INVALID; }
  if (c->initial_guess < 0 || c->initial_guess > 2) { err = "initial_guess must be 0, 1 or 2"; return IRK_ERR_INVALID; }
  if (c->mg_precision < 0 || c->mg_precision > 2) { err = "mg_precision must be 0..2"; return IRK_ERR_INVALID; }
  if (c->mg_pre < 1 || c->mg_post < 0 || c->mg_pre > 8 || c->mg_post > 8) { err = "mg sweeps out of range"; return IRK_ERR_INVALID; }
  if (c->mg_coarse_sweeps < 1 || c->mg_coarse_sweeps > 1000) { err = "mg_coarse_sweeps out of range"; return IRK_ERR_INVALID; }
  if (c->mg_shifted_sweeps < 0 || c->mg_shifted_sweeps > 8) { err = "mg_shifted_sweeps out of range"; return IRK_ERR_INVALID; }
  if (!(c->mg_coarse_reduction >= 0 && c->mg_coarse_reduction < 1)) { err = "mg_coarse_reduction must be in [0, 1)"; return IRK_ERR_INVALID; }
  if (c->mg_coarse_smoother < 0 || c->mg_coarse_smoother > 2) { err = "mg_coarse_smoother must be 0..2"; return IRK_ERR_INVALID; }
  if (c->mg_tile_rows != 0 && c->mg_tile_rows != 8 && c->mg_tile_rows != 16) { err = "mg_tile_rows must be 0, 8 or 16"; return IRK_ERR_INVALID; }
  if (c->mg_fuse_transfer < 0 || c->mg_fuse_transfer > 2) { err = "mg_fuse_transfer must be 0, 1 or 2"; return IRK_ERR_INVALID; }
  if (c->mg_levels < 0 || c->mg_levels > IRK_MAX_LEVELS) { err = "mg_levels out of range"; return IRK_ERR_INVALID; }
  return IRK_OK;
}

// Configuration of the single-stage solver of a stage-by-stage SDIRK handle:
// the same operator, grid and solver settings with one stage (its tableau,
// A = [gamma], replaces the family's).
irk_config stage_solver_config(const irk_config& c) {
  irk_config ic = c;
  ic.family = IRK_SDIRK;
  ic.stages = 1;
  ic.basis = IRK_BASIS_SCHUR;
  ic.dirk_sequential = 0;
  return ic;
}

// Plan the solver for h->cfg (tableau, grid, combined fields, MG levels,
// arena size); unless plan_only, then place the arena (the caller's when
// h->ext_arena is set, else one cudaMalloc), carve it and load u0.
irk_status build(irk_handle* h, const double* u0, int u0_on_device, bool plan_only = false) {
  const irk_config& c = h->cfg;
  char ebuf[256] = {0};
  if (h->inner_gamma > 0) {
    if (build_tableau_single(h->inner_gamma, &h->tab)) { h->err = "single-stage gamma must be positive"; return IRK_ERR_INVALID; }
  } else if (build_tableau(c.family, c.stages, c.basis, &h->tab, ebuf, sizeof ebuf)) {
    h->err = ebuf;
    return IRK_ERR_INVALID;
  }
  const int s = h->s = c.stages;
  h->dim = (c.op == IRK_OP_BURGERS_2D || c.op == IRK_OP_VSF_2D) ? 2 : 1;
  h->C = (h->dim == 2) ? 2 : 1;
  h->npts = (h->dim == 2) ? c.n * c.n : c.n;
  h->L = (long long)h->C * h->npts;
  GridDesc& g = h->g;
  g.dim = h->dim;
  g.n = c.n;
  g.logn = 0;
  while ((1 << g.logn) < c.n) ++g.logn;
  g.npts = h->npts;
  g.ncomp = h->C;
  g.op = c.op;
  g.h = c.length / c.n;
  g.inv2h = 0.5 / g.h;
  g.inv4h = 0.25 / g.h;
  g.invh2 = 1.0 / (g.h * g.h);
  g.inv12h2 = 1.0 / (12.0 * g.h * g.h);
  g.nu = c.nu;
  for (int k = 0; k < h->tab.nblk; ++k)
    for (int i = 0; i < h->tab.bsize[k]; ++i) h->blk_of[h->tab.bstart[k] + i] = k;
  // combined fields needed by the kept pattern
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) h->combo_of[i][j] = -1;
  h->ncombo = 0;
  // Block (k,l) of the transformed Jacobian (T^{-1} (x) I) diag(J(Y_m)) (T (x) I)
  // (Eq. Q0approx) is sum_m d_klm J(Y_m) with d_klm = (T^{-1})_km T_ml; each
  // kept block gets one combined field sum_m d_klm Y_m (N is bilinear).
  for (int k = 0; k < s; ++k)
    for (int l = 0; l < s; ++l) {
      const int v = std::min(c.nonlinear_variant, 3);  // variant 4 preconditions with 3
      if (!(k == l || (v >= 3 && h->blk_of[k] <= h->blk_of[l]))) continue;
      double d[IRK_MAXS], dmax = 0;
      for (int mm = 0; mm < s; ++mm) {
        d[mm] = h->tab.Tinv[k * s + mm] * h->tab.T[mm * s + l];
        dmax = std::max(dmax, std::fabs(d[mm]));
      }
      if (k != l && dmax < 1e-15) continue;
      if (v <= 1) {
        // 0: one stage for all blocks (simplified Newton); 1: the stage of the
        // largest |d_kk| entry (lumped).  Unit d-vectors keep sum_m d = 1.
        int pick = s - 1;
        if (v == 1)
          for (int mm = 0; mm < s; ++mm)
            if (std::fabs(d[mm]) > std::fabs(d[pick]) + 1e-15) pick = mm;
        for (int mm = 0; mm < s; ++mm) d[mm] = (mm == pick) ? 1.0 : 0.0;
      }
      int q = -1;
      for (int e = 0; e < h->ncombo && q < 0; ++e)
        if (std::equal(d, d + s, h->Dq + e * s)) q = e;
      if (q < 0) {
        q = h->ncombo++;
        std::copy(d, d + s, h->Dq + q * s);
      }
      h->combo_of[k][l] = q;
    }
  // multigrid levels
  h->prec = c.mg_precision;
  h->esz = mg_elem_size(h->prec);
  h->mg_omega = c.mg_omega > 0 ? c.mg_omega : (h->dim == 2 ? 0.8 : 2.0 / 3.0);
  h->mg_kind = 0;
  {
    int n = c.n, l = 0;
    const int coarsest = 8;
    while (true) {
      MGLevel& lv = h->lev[l];
      lv.d.n = n;
      lv.d.logn = 0;
      while ((1 << lv.d.logn) < n) ++lv.d.logn;
      lv.d.npts = (h->dim == 2) ? n * n : n;
      lv.d.h = c.length / n;
      ++l;
      if (n <= coarsest || l == IRK_MAX_LEVELS || (c.mg_levels > 0 && l == c.mg_levels)) break;
      n >>= 1;
    }
    h->nlev = l;
  }
  h->m = c.krylov_restart;
  // arena size
  const int maxbs = 2;
  const long long Lb = maxbs * h->L;
  size_t bytes = 0;
  auto add = [&](size_t b) { bytes += (b + 255) & ~(size_t)255; };
  add(8 * h->L);                 // u
  add(8 * h->L);                 // u_save
  add(8 * h->L * s);             // K
  add(8 * h->L * s);             // Y
  add(8 * h->L * s);             // rhs
  add(8 * h->L * s);             // yhat
  add(8 * h->L * std::max(h->ncombo, 1));  // combos
  const int ncf = combo_coef_fields(c.op);
  // coefficient fields for the combined fields of the diagonal blocks
  h->coef_list.n = 0;
  for (int q = 0; q < IRK_MAX_COMBOS; ++q) h->coef_slot[q] = -1;
  if (ncf > 0)
    for (int k = 0; k < s; ++k)
      for (int l = 0; l < s; ++l) {
        const int q = h->combo_of[k][l];
        if (q >= 0 && h->blk_of[k] == h->blk_of[l] && h->coef_slot[q] < 0) {
          h->coef_slot[q] = h->coef_list.n;
          h->coef_list.idx[h->coef_list.n++] = q;
        }
      }
  const bool use_coef = (h->coef_list.n > 0);
  if (use_coef) add(8 * (size_t)h->npts * ncf * h->coef_list.n);  // coefficient fields
  add(8 * Lb);                   // zbuf
  add(8 * h->L);                 // tmp
  add(8 * h->L);                 // tmp2
  add(8 * Lb * (h->m + 1));      // V
  add(8 * Lb * h->m);            // Z
  add(8 * Lb);                   // w
  add(8 * Lb);                   // prec_in
  add(8 * Lb);                   // prec_out
  add(sizeof(FGState) * h->tab.nblk);  // device FGMRES states
  if (h->dim == 2) add(8 * 64 * 64);  // bottom solve of the Poisson cycles
  const long long Lo = (long long)s * h->L;
  h->mo = (c.nonlinear_variant == 4) ? h->m : 0;
  if (h->mo) {
    add(8 * Lo * (h->mo + 1));   // Vo
    add(8 * Lo * h->mo);         // Zo
    for (int k = 0; k < 4; ++k) add(8 * Lo);  // wo, xo, fo, jw
  }
  h->nparts = std::max(blas_blocks(Lb) * 70, residual_blocks(g)) + 1024;
  add(8 * (size_t)h->nparts);    // partials
  add(8 * 512);                  // device scalars
  h->use_pre = (h->prec == IRK_MG_FP64 && h->dim == 2);
  for (int l = 0; l < h->nlev; ++l) {
    const size_t f = h->esz * (size_t)h->lev[l].d.npts;
    add(f * h->C); add(f * h->C); add(f * h->C); add(f * h->C);
    if (l >= 1) { add(f * h->C); add(f * h->C); }
    const size_t fv = mg_vel_size(h->prec) * (size_t)h->lev[l].d.npts;
    for (int k = 0; k < s; ++k) add(fv * h->dim);
    if (h->use_pre)
      for (int k = 0; k < s; ++k) add(f * 4);
  }
  h->arena_bytes = bytes + 4096;
  // stage-by-stage SDIRK: the single-stage solver's arena follows this one's
  h->inner_bytes = 0;
  if (c.family == IRK_SDIRK && c.dirk_sequential == 1 && s > 1 && h->inner_gamma == 0) {
    irk_handle plan;
    plan.cfg = stage_solver_config(c);
    plan.inner_gamma = h->tab.A[0];
    TRY(build(&plan, nullptr, 0, true));
    h->inner_bytes = plan.arena_bytes;
    h->arena_bytes += h->inner_bytes + 256;
  }
  if (plan_only) return IRK_OK;
  if (h->ext_arena) {
    if (h->ext_bytes < h->arena_bytes) {
      h->err = "caller-provided arena is smaller than irk_config_device_bytes()";
      return IRK_ERR_NOMEM;
    }
    h->arena = (char*)h->ext_arena;
    h->arena_bytes = h->ext_bytes;
    h->own_arena = false;
  } else {
    cudaError_t e = cudaMalloc((void**)&h->arena, h->arena_bytes);
    if (e != cudaSuccess) {
      h->arena = nullptr;
      h->err = std::string("device arena allocation failed: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return IRK_ERR_NOMEM;
    }
  }
  auto take = [&](size_t b) { return arena_take(h, b); };
  h->u = (double*)take(8 * h->L);
  h->u_save = (double*)take(8 * h->L);
  h->K = (double*)take(8 * h->L * s);
  h->Y = (double*)take(8 * h->L * s);
  h->rhs = (double*)take(8 * h->L * s);
  h->yhat = (double*)take(8 * h->L * s);
  h->combos = (double*)take(8 * h->L * std::max(h->ncombo, 1));
  h->coef = use_coef ? (double*)take(8 * (size_t)h->npts * ncf * h->coef_list.n) : nullptr;
  h->zbuf = (double*)take(8 * Lb);
  h->tmp = (double*)take(8 * h->L);
  h->tmp2 = (double*)take(8 * h->L);
  h->V = (double*)take(8 * Lb * (h->m + 1));
  h->Z = (double*)take(8 * Lb * h->m);
  h->w = (double*)take(8 * Lb);
  h->prec_in = (double*)take(8 * Lb);
  h->prec_out = (double*)take(8 * Lb);
  h->fgs = (FGState*)take(sizeof(FGState) * h->tab.nblk);
  h->pinv = (h->dim == 2) ? (double*)take(8 * 64 * 64) : nullptr;
  if (h->mo) {
    h->Vo = (double*)take(8 * Lo * (h->mo + 1));
    h->Zo = (double*)take(8 * Lo * h->mo);
    h->wo = (double*)take(8 * Lo);
    h->xo = (double*)take(8 * Lo);
    h->fo = (double*)take(8 * Lo);
    h->jw = (double*)take(8 * Lo);
  }
  h->partials = (double*)take(8 * (size_t)h->nparts);
  h->dscal = (double*)take(8 * 512);
  h->nws = h->dscal + 400;
  for (int l = 0; l < h->nlev; ++l) {
    const size_t f = h->esz * (size_t)h->lev[l].d.npts;
    h->lev[l].w = take(f * h->C);
    h->lev[l].w2 = take(f * h->C);
    h->lev[l].b = take(f * h->C);
    h->lev[l].r = take(f * h->C);
    h->lev[l].w3 = (l >= 1) ? take(f * h->C) : nullptr;
    h->lev[l].w4 = (l >= 1) ? take(f * h->C) : nullptr;
    const size_t fv = mg_vel_size(h->prec) * (size_t)h->lev[l].d.npts;
    for (int k = 0; k < s; ++k) h->vel[k][l] = take(fv * h->dim);
    for (int k = 0; k < s; ++k) h->coefh[k][l] = h->use_pre ? take(f * 4) : nullptr;
  }
  for (int k = s; k < IRK_MAXS; ++k)
    for (int l = 0; l < IRK_MAX_LEVELS; ++l) h->vel[k][l] = nullptr;
  h->inner_arena = h->inner_bytes ? take(h->inner_bytes) : nullptr;
  if (!h->dscal || (h->inner_bytes && !h->inner_arena)) { h->err = "arena layout overflow"; return IRK_ERR_NOMEM; }
  CK(cudaMemsetAsync(h->arena, 0, h->arena_used, h->st));
  CK(cudaMallocHost((void**)&h->hbuf, 4096));
  if (h->pinv) {
    // A^+ = sum over the nonzero Fourier modes k of v_k v_k^T / lambda_k, with
    // lambda_k = (4 - 2 cos(2 pi kx/8) - 2 cos(2 pi ky/8)) / h^2 on the 8^2 level
    std::vector<double> pv(64 * 64);
    const long double h8 = (long double)c.length / 8, pi = 3.14159265358979323846264338327950288L;
    for (int pp = 0; pp < 64; ++pp)
      for (int qq = 0; qq < 64; ++qq) {
        const int dx = (pp % 8) - (qq % 8), dy = (pp / 8) - (qq / 8);
        long double acc = 0;
        for (int ky = 0; ky < 8; ++ky)
          for (int kx = 0; kx < 8; ++kx) {
            if (kx == 0 && ky == 0) continue;
            const long double lam = (4 - 2 * std::cos(2 * pi * kx / 8) - 2 * std::cos(2 * pi * ky / 8)) / (h8 * h8);
            acc += std::cos(2 * pi * (kx * dx + ky * dy) / 8) / lam;
          }
        pv[pp * 64 + qq] = (double)(acc / 64);
      }
    CK(cudaMemcpy(h->pinv, pv.data(), sizeof(double) * 64 * 64, cudaMemcpyHostToDevice));
  }
  if (c.profile) {
    h->evpool.resize(8192);
    for (auto& ev : h->evpool) CK(cudaEventCreate(&ev));
  }
  for (int k = 0; k < P_NCLASS; ++k) {
    memset(&h->prof[k], 0, sizeof(irk_kernel_stat));
    snprintf(h->prof[k].name, sizeof h->prof[k].name, "%s", kProfNames[k]);
  }
  // initial state
  CK(cudaMemcpyAsync(h->u, u0, sizeof(double) * (c.op == IRK_OP_VSF_2D ? h->npts : h->L),
                     u0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  if (c.op == IRK_OP_VSF_2D) {
    // consistent psi: -L psi = omega (zero mean) by defect correction with the
    // Poisson V-cycle, to a relative residual of 1e-14
    // or, on fine grids, the rounding floor of -L_h psi in FP64 (about
    // 4e-16 / h^2 relative): the loop stops once a V-cycle no longer halves a
    // defect that is already below 1e-9
    launch_remove_mean(h->npts, 1, h->npts, h->u, h->partials, h->st);
    double* psi = h->u + h->npts;
    CK(cudaMemsetAsync(psi, 0, sizeof(double) * h->npts, h->st));
    double bnorm = 0;
    TRY(dev_norm(h, h->u, h->npts, &bnorm));
    const int save_prec = h->prec;
    double prev_dn = 0;
    for (int it = 0; it < 200 && bnorm > 0; ++it) {
      // defect d = omega - (-L_h psi) in w
      {
        ProfScope ps(h, P_POISSON, 16.0 * h->npts, 6.0 * h->npts);
        launch_neg_laplacian(h->g, psi, h->w, h->st);
      }
      launch_axpby(h->w, 1.0, h->u, -1.0, h->npts, h->st);
      double dn = 0;
      TRY(dev_norm(h, h->w, h->npts, &dn));
      if (dn <= 1e-14 * bnorm) break;
      if (it > 0 && dn > 0.5 * prev_dn && dn <= 1e-9 * bnorm) break;
      prev_dn = dn;
      h->prec = IRK_MG_FP64;
      vcycle(h, -1, MG_DIFFUSION, 1, 0.0, 0.0, 1.0, 1, h->w, h->tmp);
      h->prec = save_prec;
      launch_axpby(psi, 1.0, h->tmp, 1.0, h->npts, h->st);
    }
    h->prec = save_prec;
    h->stats.vcycles = 0;
    h->stats.poisson_vcycles = 0;
  }
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

}  // namespace

// ===========================================================================
// C ABI
#ifdef IRK_BOUNDS
long long irk::bounds_collect(std::string* msg) {
  struct Tu { const char* file; int (*take)(BoundsRecord*); };
  const Tu tus[] = {{"stencil.cu", bounds_take_stencil}, {"mg.cu", bounds_take_mg},
                    {"blas.cu", bounds_take_blas}, {"fgmres_dev.cu", bounds_take_fgmres},
                    {"noalloc.cu", bounds_take_noalloc}};
  long long total = 0;
  for (const Tu& tu : tus) {
    BoundsRecord r;
    if (tu.take(&r) != 0) return -1;
    if (r.hits != 0u && total == 0 && msg) {
      char buf[200];
      snprintf(buf, sizeof buf, "index %lld outside [0, %lld) at %s:%d (%u hits)", r.index,
               r.extent, tu.file, r.line, r.hits);
      *msg = buf;
    }
    total += r.hits;
  }
  return total;
}

// After a step: any recorded hit fails it (the caller restores the state).
static irk_status bounds_status(irk_handle* h) {
  CK(cudaStreamSynchronize(h->st));
  std::string m;
  const long long hits = bounds_collect(&m);
  if (hits == 0) return IRK_OK;
  h->err = hits < 0 ? std::string("bounds records could not be read") : "bounds check: " + m;
  return IRK_ERR_CUDA;
}
#endif

extern "C" {

void irk_config_default(irk_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->family = IRK_GAUSS;
  c->stages = 2;
  c->op = IRK_OP_BURGERS_1D;
  c->mass = IRK_MASS_IDENTITY;
  c->n = 256;
  c->length = 1.0;
  c->nu = 0.01;
  c->forcing = 0;
  c->newton_rtol = 1e-10;
  c->newton_maxit = 20;
  c->krylov_rtol = 1e-3;
  c->krylov_restart = 30;
  c->krylov_maxit = 200;
  // 2 needs the same Newton and Krylov counts as 3 on the 2D Burgers (s = 3)
  // and VSF (s = 5) workloads at 16-30% less time per step (fewer combined and
  // coefficient fields); for s = 2 Gauss and SDIRK the two coincide
  c->nonlinear_variant = 2;
  c->gamma_mode = 0;
  c->mg_precision = IRK_MG_FP64;
  c->mg_levels = 0;
  c->mg_pre = 2;
  c->mg_post = 2;
  c->mg_coarse_sweeps = 40;
  c->mg_shifted_sweeps = 1;
  c->mg_coarse_reduction = 2e-2;
  c->mg_coarse_smoother = 0;
  c->mg_omega = 0.0;
  c->profile = 0;
  c->use_graphs = 1;
  c->initial_guess = 2;
  c->dirk_sequential = 1;
  c->dae_solver = 0;
  c->mg_fuse_transfer = 0;
}

const char* irk_status_string(irk_status st) {
  switch (st) {
    case IRK_OK: return "ok";
    case IRK_ERR_INVALID: return "invalid argument";
    case IRK_ERR_NOMEM: return "out of memory";
    case IRK_ERR_CUDA: return "CUDA error";
    case IRK_ERR_NEWTON_DIVERGED: return "Newton diverged";
    case IRK_ERR_NEWTON_MAXIT: return "Newton iteration limit";
    case IRK_ERR_KRYLOV_BREAKDOWN: return "Krylov breakdown";
    case IRK_ERR_TIMEOUT: return "device wait timed out";
    case IRK_ERR_NO_DEVICE: return "no CUDA device";
  }
  return "unknown status";
}

irk_status irk_tableau(int family, int s, double* A, double* b, double* c, double* Q0, double* R0,
                       int* block_sizes, int* nblocks) {
  HostTableau t;
  char ebuf[256];
  if (build_tableau(family, s, IRK_BASIS_SCHUR, &t, ebuf, sizeof ebuf)) return IRK_ERR_INVALID;
  for (int i = 0; i < s * s; ++i) {
    if (A) A[i] = t.A[i];
    if (Q0) Q0[i] = t.T[i];
    if (R0) R0[i] = t.R[i];
  }
  for (int i = 0; i < s; ++i) {
    if (b) b[i] = t.b[i];
    if (c) c[i] = t.c[i];
  }
  if (block_sizes)
    for (int k = 0; k < t.nblk; ++k) block_sizes[k] = t.bsize[k];
  if (nblocks) *nblocks = t.nblk;
  return IRK_OK;
}

irk_status irk_transform(int family, int s, int basis, double* T, double* Tinv, double* R,
                         int* block_sizes, int* nblocks) {
  HostTableau t;
  char ebuf[256];
  if (build_tableau(family, s, basis, &t, ebuf, sizeof ebuf)) return IRK_ERR_INVALID;
  for (int i = 0; i < s * s; ++i) {
    if (T) T[i] = t.T[i];
    if (Tinv) Tinv[i] = t.Tinv[i];
    if (R) R[i] = t.R[i];
  }
  if (block_sizes)
    for (int k = 0; k < t.nblk; ++k) block_sizes[k] = t.bsize[k];
  if (nblocks) *nblocks = t.nblk;
  return IRK_OK;
}

static irk_status create_impl(const irk_config* cfg, const double* u0, int u0_on_device,
                              void* cuda_stream, void* arena, size_t arena_bytes,
                              irk_handle** out, double inner_gamma = 0.0) {
  TraceRange tr("irk_create");
  if (!out) { g_create_error = "null output handle"; return IRK_ERR_INVALID; }
  *out = nullptr;
  std::string verr;
  irk_status vs = validate(cfg, verr);
  if (vs != IRK_OK) { g_create_error = verr; return vs; }
  if (!u0) { g_create_error = "null initial state"; return IRK_ERR_INVALID; }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    g_create_error = "no CUDA device";
    return IRK_ERR_NO_DEVICE;
  }
  irk_handle* h = new (std::nothrow) irk_handle();
  if (!h) { g_create_error = "host allocation failed"; return IRK_ERR_NOMEM; }
  h->cfg = *cfg;
  h->ext_arena = arena;
  h->ext_bytes = arena_bytes;
  h->inner_gamma = inner_gamma;
  memset(&h->stats, 0, sizeof(h->stats));
  cudaGetDevice(&h->device);
  if (cuda_stream) {
    h->st = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
      g_create_error = "stream creation failed";
      delete h;
      return IRK_ERR_CUDA;
    }
    h->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&h->st_aux, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->st_aux = nullptr;  // device-resident FGMRES unavailable; host loop is used
  }
  if (cudaStreamCreateWithFlags(&h->st_aux2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->st_aux2 = nullptr;  // whole-step graph unavailable
  }
  irk_status st = build(h, u0, u0_on_device);
  if (st != IRK_OK) {
    g_create_error = h->err;
    irk_destroy(h);
    return st;
  }
  if (h->inner_arena) {
    // the stage solver shares the stream and lives in this handle's arena
    const irk_config ic = stage_solver_config(h->cfg);
    st = create_impl(&ic, h->u, 1, (void*)h->st, h->inner_arena, h->inner_bytes, &h->inner,
                     h->tab.A[0]);
    if (st != IRK_OK) {
      g_create_error = "stage solver: " + g_create_error;
      irk_destroy(h);
      return st;
    }
  }
  *out = h;
  return IRK_OK;
}

irk_status irk_create(const irk_config* cfg, const double* u0, int u0_on_device, void* cuda_stream,
                      irk_handle** out) {
  return create_impl(cfg, u0, u0_on_device, cuda_stream, nullptr, 0, out);
}

irk_status irk_create_in(const irk_config* cfg, const double* u0, int u0_on_device,
                         void* cuda_stream, void* arena, size_t arena_bytes, irk_handle** out) {
  if (!arena) { g_create_error = "null arena"; return IRK_ERR_INVALID; }
  if ((reinterpret_cast<uintptr_t>(arena) & 255) != 0) {
    g_create_error = "arena must be 256-byte aligned";
    return IRK_ERR_INVALID;
  }
  return create_impl(cfg, u0, u0_on_device, cuda_stream, arena, arena_bytes, out);
}

size_t irk_config_device_bytes(const irk_config* cfg) {
  std::string verr;
  if (validate(cfg, verr) != IRK_OK) return 0;
  irk_handle tmp;
  tmp.cfg = *cfg;
  if (build(&tmp, nullptr, 0, true) != IRK_OK) return 0;
  return tmp.arena_bytes;
}

irk_status irk_step(irk_handle* h, double t_n, double dt, int nsteps, irk_stats* stats) {
  if (!h) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0 || !std::isfinite(t_n)) {
    h->err = "dt must be positive and finite, nsteps >= 0";
    return IRK_ERR_INVALID;
  }
  TraceRange tr("irk_step");
  memset(&h->stats, 0, sizeof(h->stats));
  irk_status st = IRK_OK;
  double t = t_n;
  for (int k = 0; k < nsteps; ++k) {
    TraceRange trs("step");
    cudaError_t e = cudaMemcpyAsync(h->u_save, h->u, sizeof(double) * h->L,
                                    cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); st = IRK_ERR_CUDA; break; }
    if (h->inner) {
      st = sdirk_sequential_step(h, t, dt);
    } else {
      st = prepare_guess(h, dt);
      if (st == IRK_OK) {
        st = graph_step(h, dt);
        if (st == IRK_ERR_INVALID) st = newton_step(h, t, dt);  // host-driven loop
      }
    }
#ifdef IRK_BOUNDS
    if (st == IRK_OK) st = bounds_status(h);
#endif
    if (st != IRK_OK) {
      cudaMemcpyAsync(h->u, h->u_save, sizeof(double) * h->L, cudaMemcpyDeviceToDevice, h->st);
      cudaMemsetAsync(h->K, 0, sizeof(double) * h->L * h->s, h->st);  // discard the failed iterate
      cudaStreamSynchronize(h->st);
      h->last_dt = 0.0;
      break;
    }
    h->last_dt = dt;
    h->stats.steps += 1;
    t += dt;
  }
  if (st == IRK_OK) {
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); st = IRK_ERR_CUDA; }
  }
  prof_harvest(h);
  if (h->inner) prof_harvest(h->inner);
  if (stats) *stats = h->stats;
  return st;
}

irk_status irk_get_state(irk_handle* h, double* dst, int dst_on_device) {
  if (!h || !dst) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  CK(cudaMemcpyAsync(dst, h->u, sizeof(double) * h->L,
                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

irk_status irk_set_state(irk_handle* h, const double* src, int src_on_device) {
  if (!h || !src) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  CK(cudaMemcpyAsync(h->u, src, sizeof(double) * h->L,
                     src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  // a new state starts Newton from zero stages
  CK(cudaMemsetAsync(h->K, 0, sizeof(double) * h->L * h->s, h->st));
  h->last_dt = 0.0;
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

irk_status irk_set_state_keep_stages(irk_handle* h, const double* src, int src_on_device) {
  if (!h || !src) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  CK(cudaMemcpyAsync(h->u, src, sizeof(double) * h->L,
                     src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

irk_status irk_set_stages(irk_handle* h, const double* src, int src_on_device) {
  if (!h || !src) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  CK(cudaMemcpyAsync(h->K, src, sizeof(double) * h->L * h->s,
                     src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  h->last_dt = -1.0;  // the caller's stages: taken as from a step of the next step's dt
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

irk_status irk_get_stages(irk_handle* h, double* dst, int dst_on_device) {
  if (!h || !dst) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  CK(cudaMemcpyAsync(dst, h->K, sizeof(double) * h->L * h->s,
                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

irk_status irk_stage_residual(irk_handle* h, double t_n, double dt, const double* K, double* F,
                              int on_device) {
  if (!h || !K || !F) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  TraceRange tr("irk_stage_residual");
  const size_t bytes = sizeof(double) * h->L * h->s;
  // stage the input in yhat (free between steps) and the output in rhs
  CK(cudaMemcpyAsync(h->yhat, K, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  double fn = 0;
  TRY(eval_residual(h, t_n, dt, h->yhat, nullptr, h->rhs, false, &fn));
  CK(cudaMemcpyAsync(F, h->rhs, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  prof_harvest(h);
#ifdef IRK_BOUNDS
  TRY(bounds_status(h));
#endif
  return IRK_OK;
}

irk_status irk_stage_jacobian_apply(irk_handle* h, double dt, const double* K, const double* V,
                                    double* JV, int on_device) {
  if (!h || !K || !V || !JV) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  TraceRange tr("irk_stage_jacobian_apply");
  const int s = h->s;
  const size_t bytes = sizeof(double) * h->L * s;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // K -> yhat, V -> V-basis scratch, W_i = sum_j a_ij v_j -> combos region is not used here
  double* Kd = h->yhat;
  double* Vd = h->V;
  double* Wd = h->V + (long long)s * h->L;
  double* Out = h->rhs;
  if ((long long)2 * s * h->L > (long long)2 * h->L * (h->m + 1)) { h->err = "restart too small for the Jacobian scratch"; return IRK_ERR_INVALID; }
  CK(cudaMemcpyAsync(Kd, K, bytes, kin, h->st));
  CK(cudaMemcpyAsync(Vd, V, bytes, kin, h->st));
  StageStateArgs sa;
  set_stage_args(h, sa, dt, h->u, Kd, h->Y, nullptr);
  launch_stage_states(h->g, sa, h->st);
  full_jvp(h, dt, Vd, Out, Wd);
  CK(cudaMemcpyAsync(JV, Out, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  prof_harvest(h);
#ifdef IRK_BOUNDS
  TRY(bounds_status(h));
#endif
  return IRK_OK;
}

// Drop every captured graph (L_P, block solves, whole step): the next step
// captures again with the handle's current settings.
static void invalidate_graphs(irk_handle* h) {
  drop_graphs(h);
  h->graph_dt = 0.0;
  drop_fg_graphs(h);
  h->fg_dt = 0.0;
  for (int k = 0; k < IRK_MAXS; ++k) h->fg_seen_its[k] = 0.0;
  if (h->stepexec) {
    cudaGraphExecDestroy(h->stepexec);
    h->stepexec = nullptr;
  }
  h->step_dt = 0.0;
}

irk_status irk_get_config(const irk_handle* h, irk_config* out) {
  if (!h || !out) return IRK_ERR_INVALID;
  *out = h->cfg;
  return IRK_OK;
}

irk_status irk_autotune(irk_handle* h, double t_n, double dt, int steps, irk_config* chosen) {
  if (!h || !(dt > 0) || !std::isfinite(dt) || steps < 1 || steps > 100 || !std::isfinite(t_n)) {
    if (h) h->err = "autotune: dt must be positive, 1 <= steps <= 100";
    return IRK_ERR_INVALID;
  }
  DeviceScope ds(h->device);
  TraceRange tr("irk_autotune");
  const size_t ub = sizeof(double) * h->L, kb = sizeof(double) * h->L * h->s;
  double *u0 = nullptr, *k0 = nullptr;
  cudaError_t e = cudaMalloc((void**)&u0, ub);
  if (e == cudaSuccess) e = cudaMalloc((void**)&k0, kb);
  if (e != cudaSuccess) {
    cudaFree(u0);
    cudaGetLastError();
    h->err = "autotune: no device memory for the state backup";
    return IRK_ERR_NOMEM;
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  irk_status st = IRK_OK;
  const irk_stats saved_stats = h->stats;
  auto restore = [&]() -> irk_status {
    CK(cudaMemcpyAsync(h->u, u0, ub, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->K, k0, kb, cudaMemcpyDeviceToDevice, h->st));
    return IRK_OK;
  };
  // ms per step of the current settings from the saved state (one untimed
  // step first: it captures the graphs), or +inf when a step fails
  auto measure = [&](double* ms) -> irk_status {
    invalidate_graphs(h);
    if (h->inner) {
      // the stage solver of a stage-by-stage SDIRK handle runs the V-cycles
      h->inner->cfg.mg_shifted_sweeps = h->cfg.mg_shifted_sweeps;
      h->inner->cfg.mg_coarse_smoother = h->cfg.mg_coarse_smoother;
      h->inner->cfg.mg_coarse_reduction = h->cfg.mg_coarse_reduction;
      h->inner->cfg.mg_tile_rows = h->cfg.mg_tile_rows;
      h->inner->cfg.mg_levels = h->cfg.mg_levels;
      h->inner->cfg.mg_fuse_transfer = h->cfg.mg_fuse_transfer;
      invalidate_graphs(h->inner);
    }
    TRY(restore());
    *ms = INFINITY;
    if (irk_step(h, t_n, dt, 1, nullptr) != IRK_OK) return IRK_OK;
    TRY(restore());
    CK(cudaEventRecord(ev0, h->st));
    const irk_status r = irk_step(h, t_n, dt, steps, nullptr);
    CK(cudaEventRecord(ev1, h->st));
    CK(cudaEventSynchronize(ev1));
    if (r != IRK_OK) return IRK_OK;
    float t = 0;
    CK(cudaEventElapsedTime(&t, ev0, ev1));
    *ms = t / steps;
    return IRK_OK;
  };
  do {
    e = cudaMemcpyAsync(u0, h->u, ub, cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(k0, h->K, kb, cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); st = IRK_ERR_CUDA; break; }
    double best = 0;
    st = measure(&best);
    if (st != IRK_OK) break;
    // coordinate descent over the multigrid knobs of the V-cycle preconditioner:
    // sweeps on shift-dominated rows, the coarsest-level smoother and its
    // target, the tile height of the three-sweep kernel, and the V-cycle
    // depth (the automatic depth of the first row against one level deeper),
    // and the fused residual-restriction kernel against the two kernels
    struct Knob { int which; double vals[2]; };
    const int d0 = mg_depth(h, row_shift(h, 0), dt * h->g.nu);
    const double deeper = (h->cfg.mg_levels == 0 && d0 + 1 <= h->nlev) ? d0 + 1 : 0;
    const int auto_rows = (h->prec == IRK_MG_FP64) ? 16 : 8;
    const int auto_fuse = (h->prec == IRK_MG_FP64) ? 2 : 1;
    const Knob knobs[6] = {{0, {1, 2}}, {1, {0, 2}}, {2, {2e-2, 5e-3}}, {3, {8, 16}},
                           {4, {0, deeper}}, {5, {1, 2}}};
    for (const Knob& kn : knobs) {
      for (double v : kn.vals) {
        irk_config trial = h->cfg;
        if (kn.which == 0) { if (trial.mg_shifted_sweeps == (int)v) continue; trial.mg_shifted_sweeps = (int)v; }
        if (kn.which == 1) { if (trial.mg_coarse_smoother == (int)v) continue; trial.mg_coarse_smoother = (int)v; }
        if (kn.which == 2) { if (trial.mg_coarse_reduction == v) continue; trial.mg_coarse_reduction = v; }
        if (kn.which == 3) {
          const int now = trial.mg_tile_rows ? trial.mg_tile_rows : auto_rows;
          if (now == (int)v) continue;
          trial.mg_tile_rows = (int)v;
        }
        if (kn.which == 4) { if (trial.mg_levels == (int)v) continue; trial.mg_levels = (int)v; }
        if (kn.which == 5) {
          const int now = trial.mg_fuse_transfer ? trial.mg_fuse_transfer : auto_fuse;
          if (now == (int)v) continue;
          trial.mg_fuse_transfer = (int)v;
        }
        const irk_config keep = h->cfg;
        h->cfg = trial;
        double ms = 0;
        st = measure(&ms);
        if (st != IRK_OK) break;
        if (ms < best) best = ms;
        else h->cfg = keep;
      }
      if (st != IRK_OK) break;
    }
  } while (0);
  invalidate_graphs(h);
  if (st == IRK_OK) st = restore();
  cudaStreamSynchronize(h->st);
  h->stats = saved_stats;
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaFree(u0);
  cudaFree(k0);
  if (chosen) *chosen = h->cfg;
  return st;
}

irk_status irk_kernel_stats(irk_handle* h, irk_kernel_stat* out, int max, int* count) {
  if (!h || !out || !count) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  prof_harvest(h);
  if (h->inner) prof_harvest(h->inner);
  int n = 0;
  for (int k = 0; k < P_NCLASS && n < max; ++k) {
    irk_kernel_stat ks = h->prof[k];
    if (h->inner) {  // the stage solver's launches of the same class
      const irk_kernel_stat& q = h->inner->prof[k];
      ks.launches += q.launches;
      ks.ms += q.ms;
      ks.bytes += q.bytes;
      ks.flops += q.flops;
    }
    if (ks.launches > 0) out[n++] = ks;
  }
  *count = n;
  return IRK_OK;
}

irk_status irk_reset_kernel_stats(irk_handle* h) {
  if (!h) return IRK_ERR_INVALID;
  DeviceScope ds(h->device);
  prof_harvest(h);
  for (int k = 0; k < P_NCLASS; ++k) {
    h->prof[k].launches = 0;
    h->prof[k].ms = h->prof[k].bytes = h->prof[k].flops = 0;
  }
  if (h->inner) irk_reset_kernel_stats(h->inner);
  return IRK_OK;
}

size_t irk_device_bytes(const irk_handle* h) { return h ? h->arena_bytes : 0; }

const char* irk_last_error(const irk_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void irk_destroy(irk_handle* h) {
  if (!h) return;
  DeviceScope ds(h->device);
  if (h->inner) irk_destroy(h->inner);
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto& ev : h->evpool) cudaEventDestroy(ev);
  if (h->hbuf) cudaFreeHost(h->hbuf);
  for (int k = 0; k < IRK_MAXS; ++k)
    if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
  for (int k = 0; k < IRK_MAXS; ++k)
    if (h->fgexec[k]) cudaGraphExecDestroy(h->fgexec[k]);
  if (h->stepexec) cudaGraphExecDestroy(h->stepexec);
  if (h->st_aux) cudaStreamDestroy(h->st_aux);
  if (h->st_aux2) cudaStreamDestroy(h->st_aux2);
  if (h->arena && h->own_arena) cudaFree(h->arena);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
}

long long irk_debug_bounds(int selftest, char* msg, size_t msg_len) {
  std::string m;
  long long hits = -1;
#ifdef IRK_BOUNDS
  if (selftest) {
    launch_bounds_selftest(0);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      m = "self-test launch failed";
      hits = -2;
    }
  }
  if (hits != -2) {
    hits = bounds_collect(&m);
    if (hits < 0) {
      hits = -2;
      m = "bounds records could not be read";
    }
  }
#else
  (void)selftest;
  m = "not a bounds-checked build";
#endif
  if (msg && msg_len > 0) snprintf(msg, msg_len, "%s", m.c_str());
  return hits;
}

}  // extern "C"
