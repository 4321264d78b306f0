// Batched Gauss-IRK stage solve (include/irk_batch.h): many independent 2D
// viscous Burgers problems of different sizes advanced in lock step, each
// kernel launch covering all of them.
//
// Every kernel here is a persistent launch of kGrid CTAs that walks a plan:
// a list of tasks (one per instance, per block solve or per multigrid row
// taking part in the phase), each split into chunks of consecutive work
// items; CTA c takes chunks c, c + kGrid, ...  and finds the owning task by
// a binary search over the chunk starts.  A chunk belongs to one task, so a
// per-task reduction is the fixed-order sum of that task's chunk partials,
// independent of the other tasks in the launch: an instance computes the
// same numbers bit for bit alone and in any mix.
//
// One step (Algorithm 1 of Sec. 5 per instance, Newton-like variant 2 of
// Sec. 3.2) is one CUDA graph:
//   prefix    u_save = u; K <- extrapolated previous stages; ||F(0)||;
//             F(K); Newton test (a guess worse than zero stages: K = 0, F again)
//   WHILE     any instance iterating (Newton):
//               multigrid coefficient hierarchy of every diagonal row
//               for each round (Schur blocks from the last, back substitution):
//                 z = rhs_blk - R_{blk,later} yhat_later (mass coupling, Eq. D+U);
//                 FGMRES init; WHILE any block solve running: L_P (two
//                 V-cycle phases and the coupling row, Eq. Lprec), block
//                 operator (Eq. diag_blocks), fused CGS2 + Arnoldi/Givens;
//                 y = R^{-1} g, yhat_blk = Z y
//               K += (T R (x) I) yhat; F(K); Newton test and forcing term
//   suffix    u += dt sum_i b_i K_i (Eq. update), or K = 0 after a failure.
// Launches in which no task takes part cost one empty grid; the graph is
// captured again only when its launch sequence changes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/irk_batch.h"
#include "irk_internal.h"

namespace irk {
namespace bat {

constexpr int kThreads = 256;
constexpr int kGrid = 152 * 4;
constexpr int kMaxLev = 12;
constexpr int kPS = 32;       // partial slots per chunk: Krylov basis size + 1 <= 31 + 1
constexpr int kMaxM = 30;     // FGMRES(m) limit of the batched path
constexpr int kGsItems = 4;   // items per thread in the Krylov basis kernels
constexpr int kMaxBlk = 3;    // Schur blocks per instance (s <= 5)

enum Flag { F_NONE = 0, F_INST = 1, F_SYS = 2, F_REJ = 3 };

struct Task {
  int n, logn, npts;   // grid of the level the task works on
  int count;           // work items
  int nchunk;          // chunks of this task in the plan
  int pbase;           // first partial slot block (per chunk) of this task
  int inst, sys;       // owner instance / block solve (-1: none)
  int flag;            // Flag
  const int* flagp;    // the flag word (set by the host from flag): the task
  int on_nonzero;      // runs when (*flagp != 0) == on_nonzero
  int first;           // sweep from w = 0 (residual: of the folded sweep; prolongation: set)
  int nsw;             // damped-Jacobi sweeps of a k_bsweep task (1..3)
  int p2base, n2chunk; // Newton: the ||F(0)|| partials
  double c[6];
  const double* in[4];
  double* out[2];
};

struct Plan {
  int ntask, nchunk, task0, cs0;
};

// Read-only description of one instance.
struct Inst {
  int s, n, logn, npts;
  long long L;
  double dt, nu, h, inv2h, invh2;
  double newton_rtol, krylov_rtol;
  int newton_maxit;
  double A[IRK_MAXS * IRK_MAXS], b[IRK_MAXS], Tinv[IRK_MAXS * IRK_MAXS], TR[IRK_MAXS * IRK_MAXS];
  double R[IRK_MAXS * IRK_MAXS], E[IRK_MAXS * IRK_MAXS], Dd[IRK_MAXS * IRK_MAXS];
  double *u, *u_save, *K, *Y, *combos, *ccoef, *rhs, *yhat;
};

// Newton state of one instance (device, written by the control kernels).
struct Newton {
  double f0, fn, rel, prev, prev_rel, eta;
  int its, status, active, rejected, kits, vcyc;
};

// One block solve (instance, Schur block): FGMRES data and counters.
struct Sys {
  int inst, a, bs, m;
  long long Lb;
  double *V, *Z, *w, *pin, *pout, *tmpb;
  FGState* fs;
  unsigned int ctr0, ctr1, ctr2;
  double h1[kPS], h2[kPS];
};

struct Dev {
  const Plan* plans;
  const Task* tasks;
  const int* cs;
  const int* ctask;  // per plan and CTA: the task of chunk blockIdx.x (-1: none)
  const Inst* inst;
  Newton* nw;
  Sys* sys;
  double* partials;
  int* guard;  // per round: Krylov body executions
};

// ---------------------------------------------------------------------------
// Walk the chunks of plan pi; f(task, local chunk) runs with the whole CTA.
// The task of this CTA's first chunk comes from a per-plan table (one load,
// issued together with the plan header); later chunks belong to the same or
// later tasks, found by stepping forward through the chunk starts.
template <class F>
__device__ __forceinline__ void for_chunks(const Dev& D, int pi, F f) {
  const Plan P = D.plans[pi];
  int t = D.ctask[pi * kGrid + blockIdx.x];
  for (int c = blockIdx.x; c < P.nchunk; c += gridDim.x) {
    while (D.cs[P.cs0 + t + 1] <= c) ++t;
    const Task& tk = D.tasks[P.task0 + t];
    if (tk.flagp && ((*(volatile const int*)tk.flagp != 0) != (tk.on_nonzero != 0))) continue;
    f(tk, c - D.cs[P.cs0 + t]);
  }
}

// Sum over the CTA (fixed order); the result is valid in thread 0.
__device__ __forceinline__ double cta_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kThreads / 32; ++k) r += sh[k];
  return r;
}

// The CTA that finishes the last chunk of a task (atomic arrival count,
// reset by that CTA).
__device__ bool arrive_last(unsigned int* ctr, int total) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ctr, 1u) == (unsigned)total - 1u);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// out[v] = sum over the task's chunks of partials[chunk][v], v < count, in
// chunk order (the whole CTA; warp w sums values w, w + 8, ...)
__device__ void reduce_partials(const double* partials, int pbase, int nchunk, int count,
                                double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v = wid; v < count; v += kThreads / 32) {
    double acc = 0.0;
    for (int b = lane; b < nchunk; b += 32) acc += __ldcg(partials + (long long)(pbase + b) * kPS + v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[v] = acc;
  }
}

// the same sum for one value, by one warp (lane 0 holds it)
__device__ __forceinline__ double warp_reduce_partials(const double* partials, int pbase,
                                                       int nchunk) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int b = lane; b < nchunk; b += 32) acc += __ldcg(partials + (long long)(pbase + b) * kPS);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  return acc;
}

struct P5 {
  int c, e, w, n, s;
};
__device__ __forceinline__ P5 nbr(int p, int n, int logn) {
  const int m = n - 1, i = p & m, j = p >> logn;
  P5 r;
  r.c = p;
  r.e = (j << logn) + ((i + 1) & m);
  r.w = (j << logn) + ((i - 1) & m);
  r.n = (((j + 1) & m) << logn) + i;
  r.s = (((j - 1) & m) << logn) + i;
  return r;
}

// N of 2D Burgers at point p, component c of the state Y (u then v):
// nu L f - (u Dx f + v Dy f), as the single-instance residual kernel forms it.
__device__ __forceinline__ double burgers_n(const double* __restrict__ Y, int npts, int c,
                                            const P5& q, double nuh, double mi2h) {
  const double* f = Y + (long long)c * npts;
  const double uc = __ldg(Y + q.c), vc = __ldg(Y + npts + q.c);
  const double fc = c ? vc : uc;
  const double fe = __ldg(f + q.e), fw = __ldg(f + q.w), fn = __ldg(f + q.n), fs = __ldg(f + q.s);
  double adv = uc * (fe - fw);
  adv = fma(vc, fn - fs, adv);
  double lap = (fe + fw) + (fn + fs);
  lap = fma(-4.0, fc, lap);
  return fma(nuh, lap, mi2h * adv);
}

// ---------------------------------------------------------------------------
// Newton-level kernels (tasks: instances).  The stage count is a template
// parameter of the per-point bodies (registers, not local memory); a chunk
// belongs to one instance, so the switch on its s is uniform in the CTA.
#define IRK_BAT_STAGES(s_, CALL)          \
  switch (s_) {                           \
    case 1: { constexpr int S = 1; CALL; } break; \
    case 2: { constexpr int S = 2; CALL; } break; \
    case 3: { constexpr int S = 3; CALL; } break; \
    case 4: { constexpr int S = 4; CALL; } break; \
    default: { constexpr int S = 5; CALL; } break; \
  }

template <int S>
__device__ __forceinline__ void begin_point(const Inst& I, long long p, bool extrapolate) {
  I.u_save[p] = I.u[p];
  double k[S];
#pragma unroll
  for (int i = 0; i < S; ++i) k[i] = I.K[i * I.L + p];
#pragma unroll
  for (int j = 0; j < S; ++j) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < S; ++i) acc = fma(I.E[j * S + i], k[i], acc);
    I.K[j * I.L + p] = extrapolate ? acc : 0.0;
  }
}

template <int S>
__device__ __forceinline__ void states_point(const Inst& I, long long p) {
  const long long L = I.L;
  double k[S], y[S];
#pragma unroll
  for (int j = 0; j < S; ++j) k[j] = I.K[j * L + p];
  const double u = I.u[p];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) acc = fma(I.A[i * S + j], k[j], acc);
    y[i] = fma(I.dt, acc, u);
    I.Y[i * L + p] = y[i];
  }
#pragma unroll
  for (int q = 0; q < S; ++q) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < S; ++m) acc = fma(I.Dd[q * S + m], y[m], acc);
    I.combos[q * L + p] = acc;
  }
}

// F_i = k_i - N(Y_i) at item q (component c, point p); rhs; returns sum F_i^2
template <int S>
__device__ __forceinline__ double resid_point(const Inst& I, int q) {
  const int c = q >= I.npts ? 1 : 0, p = q - c * I.npts;
  const P5 nb = nbr(p, I.n, I.logn);
  const long long L = I.L;
  double F[S], sq = 0.0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const double nv = burgers_n(I.Y + i * L, I.npts, c, nb, I.nu * I.invh2, -I.inv2h);
    F[i] = __ldg(I.K + i * L + q) - nv;
    sq = fma(F[i], F[i], sq);
  }
#pragma unroll
  for (int k = 0; k < S; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < S; ++i) acc = fma(-I.Tinv[k * S + i], F[i], acc);
    I.rhs[k * L + q] = acc;
  }
  return sq;
}

template <int S>
__device__ __forceinline__ void update_point(const Inst& I, long long p) {
  double y[S];
#pragma unroll
  for (int k = 0; k < S; ++k) y[k] = I.yhat[k * I.L + p];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double acc = I.K[i * I.L + p];
#pragma unroll
    for (int k = 0; k < S; ++k) acc = fma(I.TR[i * S + k], y[k], acc);
    I.K[i * I.L + p] = acc;
  }
}

// u_save = u; K <- E K (c[0] = 1) or 0
__global__ void __launch_bounds__(kThreads) k_begin(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const long long p = (long long)lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    IRK_BAT_STAGES(I.s, begin_point<S>(I, p, t.c[0] != 0.0));
  });
}

// partial sums of ||N(u)||^2 (one stage of F(k = 0); every stage is equal)
__global__ void __launch_bounds__(kThreads) k_f0(Dev D, int pi) {
  __shared__ double sh[kThreads / 32];
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const int q = lc * kThreads + threadIdx.x;
    double sq = 0.0;
    if (q < t.count) {
      const int c = q >= I.npts ? 1 : 0, p = q - c * I.npts;
      const double nv = burgers_n(I.u, I.npts, c, nbr(p, I.n, I.logn), I.nu * I.invh2, -I.inv2h);
      sq = nv * nv;
    }
    const double tot = cta_sum(sq, sh);
    if (threadIdx.x == 0) D.partials[(long long)(t.pbase + lc) * kPS] = tot;
  });
}

// Y_i = u + dt sum_j a_ij k_j; diagonal combined fields Ybar_kk = sum_m Dd_km Y_m
__global__ void __launch_bounds__(kThreads) k_states(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const long long p = (long long)lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    IRK_BAT_STAGES(I.s, states_point<S>(I, p));
  });
}

// Six coefficient fields of every diagonal combined field (ub, vb) for the
// block operator: dt ub/(2h), dt vb/(2h), dt Dx ub, dt Dy ub, dt Dx vb, dt Dy vb
__global__ void __launch_bounds__(kThreads) k_ccoef(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const int p = lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    const P5 q = nbr(p, I.n, I.logn);
    const double dth = I.dt * I.inv2h;
    const int np = I.npts;
    for (int k = 0; k < I.s; ++k) {
      const double* bu = I.combos + (long long)k * I.L;
      const double* bv = bu + np;
      double* f = I.ccoef + (long long)k * 6 * np + p;
      f[0] = dth * __ldg(bu + q.c);
      f[np] = dth * __ldg(bv + q.c);
      f[2 * np] = dth * (__ldg(bu + q.e) - __ldg(bu + q.w));
      f[3 * np] = dth * (__ldg(bu + q.n) - __ldg(bu + q.s));
      f[4 * np] = dth * (__ldg(bv + q.e) - __ldg(bv + q.w));
      f[5 * np] = dth * (__ldg(bv + q.n) - __ldg(bv + q.s));
    }
  });
}

// F_i = k_i - N(Y_i); rhs_k = -sum_i (T^{-1})_ki F_i; partial ||F||^2
__global__ void __launch_bounds__(kThreads) k_resid(Dev D, int pi) {
  __shared__ double sh[kThreads / 32];
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const int q = lc * kThreads + threadIdx.x;
    double sq = 0.0;
    if (q < t.count) IRK_BAT_STAGES(I.s, sq = resid_point<S>(I, q));
    const double tot = cta_sum(sq, sh);
    if (threadIdx.x == 0) D.partials[(long long)(t.pbase + lc) * kPS] = tot;
  });
}

// K = 0 for the instances whose warm start was rejected
__global__ void __launch_bounds__(kThreads) k_reject(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const long long p = (long long)lc * kThreads + threadIdx.x;
    if (p < t.count) I.K[p] = 0.0;
  });
}

// The inexact-Newton forcing term of the single-instance solver (same rule).
__device__ double forcing(double rel, double prev_rel, double fn, double prev, int it,
                          double newton_rtol, double krylov_rtol) {
  double eta = fmin(krylov_rtol, rel);
  if (it > 0 && prev > 0.0 && fn > 0.5 * prev) eta = fmin(eta, 1e-3 * rel);
  if (it > 0 && prev_rel > 0.0 && (rel / (prev_rel * prev_rel)) * rel * rel <= 0.25 * newton_rtol)
    eta = fmin(eta, 0.5 * newton_rtol / rel);
  eta = fmax(eta, 0.2 * newton_rtol / rel);
  return fmax(eta, 1e-13);
}

enum NewtonMode { N_FIRST = 0, N_RECHECK = 1, N_CTL = 2 };

// One instance's Newton test (see k_newton); f2 = ||F||^2 of this evaluation,
// f02 = ||N(u)||^2 (FIRST only).
__device__ void newton_one(Newton& N, const Inst& I, int mode, double f2, double f02) {
    const double fn = isfinite(f2) ? sqrt(fmax(f2, 0.0)) : f2;
    if (mode == N_FIRST) {
      const double f0 = isfinite(f02) ? sqrt(fmax(I.s * f02, 0.0)) : f02;
      N.f0 = f0;
      N.its = 0;
      N.status = 0;
      N.kits = 0;
      N.vcyc = 0;
      N.rejected = 0;
      N.prev = f0;
      N.prev_rel = 0.0;
      N.active = 0;
      if (!isfinite(f0)) {
        N.status = IRK_ERR_NEWTON_DIVERGED;
        N.rel = f0;
        return;
      }
      if (f0 == 0.0) {  // zero stages solve the stage equations
        N.rejected = 1;
        N.rel = 0.0;
        N.fn = 0.0;
        return;
      }
    } else if (mode == N_RECHECK) {
      if (!N.rejected) return;
      N.rejected = 0;
      if (N.f0 == 0.0) return;
    } else if (!N.active) {
      return;
    }
    const int count = (mode == N_CTL) ? 1 : 0;
    const int it = N.its + count;
    const double rel = fn / N.f0;
    N.fn = fn;
    N.rel = rel;
    N.its = it;
    int stop = 1;
    if (!isfinite(fn)) N.status = IRK_ERR_NEWTON_DIVERGED;
    else if (rel <= I.newton_rtol) N.status = 0;
    else if (mode == N_FIRST && rel > kGuessLimit) { N.rejected = 1; stop = 2; }
    else if (it >= I.newton_maxit) N.status = IRK_ERR_NEWTON_MAXIT;
    else if (rel > 1e3) N.status = IRK_ERR_NEWTON_DIVERGED;
    else stop = 0;
    if (stop) {
      N.active = 0;
      return;
    }
    N.eta = forcing(rel, count ? N.prev_rel : 0.0, fn, N.prev, it, I.newton_rtol, I.krylov_rtol);
    N.prev = fn;
    N.prev_rel = rel;
    N.active = 1;
}

// Newton tests of every instance (one warp per instance); the WHILE condition
// is whether any instance iterates.  FIRST: ||F(0)|| (s equal stages) and the
// warm start's ||F||; a guess worse than zero stages is marked rejected.
// RECHECK: ||F|| of the rejected instances' zero stages.  CTL: after an update.
__global__ void k_newton(Dev D, int pi, int mode, cudaGraphConditionalHandle cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const Plan P = D.plans[pi];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int ti = wid; ti < P.ntask; ti += nwarp) {
    const Task& t = D.tasks[P.task0 + ti];
    Newton& N = D.nw[t.inst];
    const Inst& I = D.inst[t.inst];
    const double f2 = warp_reduce_partials(D.partials, t.pbase, t.nchunk);
    double f02 = 0.0;
    if (mode == N_FIRST) f02 = warp_reduce_partials(D.partials, t.p2base, t.n2chunk);
    if (lane != 0) continue;
    newton_one(N, I, mode, f2, f02);
    if (N.active) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && mode != N_FIRST) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

// K += (T R (x) I) yhat
__global__ void __launch_bounds__(kThreads) k_update(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const long long p = (long long)lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    IRK_BAT_STAGES(I.s, update_point<S>(I, p));
  });
}

// u_{n+1} = u_n + dt sum_i b_i k_i (Eq. update); after a failure the state
// stays and the next step starts from zero stages
__global__ void __launch_bounds__(kThreads) k_finish(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Inst& I = D.inst[t.inst];
    const long long p = (long long)lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    const Newton& N = D.nw[t.inst];
    const int s = I.s;
    if (N.status == 0) {
      double acc = 0.0;
      for (int i = 0; i < s; ++i) acc = fma(I.b[i], I.K[i * I.L + p], acc);
      I.u[p] = fma(I.dt, acc, I.u[p]);
    } else {
      for (int i = 0; i < s; ++i) I.K[i * I.L + p] = 0.0;
    }
  });
}

// ---------------------------------------------------------------------------
// Multigrid (tasks: one row and level).  Two fields per row (the u and v
// parts of a block row), one scalar operator
//   A w = sigma w + dt (a_x Dx w + a_y Dy w) - dt nu L w
// with the row's combined field as the frozen velocity a, rediscretised on
// every level, in coefficient form A w = D w_c + sum_k c_k w_k.

// full weighting of two fields: fine in[0] (grid n) -> coarse out[0]
__global__ void __launch_bounds__(kThreads) k_restrict(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const int p = lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    const int n = t.n, lf = t.logn, m = n - 1, nc = n >> 1, logc = lf - 1;
    const int I0 = p & (nc - 1), J0 = p >> logc;
    const int i = 2 * I0, j = 2 * J0;
    const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
    for (int c = 0; c < 2; ++c) {
      const double* f = t.in[0] + (long long)c * t.npts;
      const double centre = f[(j << lf) + i];
      const double edges = f[(j << lf) + ip] + f[(j << lf) + im] + f[(jp << lf) + i] + f[(jm << lf) + i];
      const double corners = f[(jp << lf) + ip] + f[(jp << lf) + im] + f[(jm << lf) + ip] +
                             f[(jm << lf) + im];
      t.out[0][(long long)c * t.count + p] = (4.0 * centre + 2.0 * edges + corners) * 0.0625;
    }
  });
}

// coefficient fields of a level from its velocity: c[0] = alpha = dt/(2h),
// c[1] = beta = -dt nu / h^2; out = (beta + alpha a_x, beta - alpha a_x,
// beta + alpha a_y, beta - alpha a_y)
__global__ void __launch_bounds__(kThreads) k_mgcoef(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const int p = lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    const double ax = t.in[0][p], ay = t.in[0][t.npts + p];
    const double al = t.c[0], be = t.c[1];
    double* o = t.out[0];
    o[p] = fma(al, ax, be);
    o[t.npts + p] = fma(-al, ax, be);
    o[2 * t.npts + p] = fma(al, ay, be);
    o[3 * t.npts + p] = fma(-al, ay, be);
  });
}

// One to three damped-Jacobi sweeps (t.nsw) of a multigrid row on one level.
// A chunk is a 32 x 8 tile (n >= 32), staged with a halo of nsw points: b,
// the iterate and the four coefficients go to shared memory once, and the
// sweeps run out of it on windows that shrink by one point per sweep; the
// last one writes the tile.  A level of n <= 16 is one chunk, held whole
// (periodic wrap in shared memory).  in[0] = b, in[1] = w (unused when
// first), in[2] = coefficients; out[0] = the new w; c[0] = omega/D,
// c[1] = 1 - omega.  Epilogue when out[1] is set (the L_P coupling row of a
// 2x2 block): out[1] = in[3] + c[2] w on the last sweep.
constexpr int kBX = 32, kBY = 8, kBH = 3;
constexpr int kBW = kBX + 2 * kBH, kBHt = kBY + 2 * kBH;
__global__ void __launch_bounds__(kThreads) k_bsweep(Dev D, int pi) {
  __shared__ double sw[2][kBHt * kBW];
  __shared__ double sb[kBHt * kBW];
  __shared__ double sc[4][kBHt * kBW];
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const int n = t.n, m = n - 1, ln = t.logn, np = t.npts, h = t.nsw;
    const double dinv = t.c[0], keep = t.c[1];
    const double* b = t.in[0];
    const double* w = t.in[1];
    const double* cf = t.in[2];
    double* wo = t.out[0];
    double* eo = t.out[1];
    const double* eb = t.in[3];
    if (n >= kBX) {
      const int tpr = n / kBX;
      const int x0 = (lc % tpr) * kBX - h, y0 = (lc / tpr) * kBY - h;
      const int W = kBX + 2 * h, H = kBY + 2 * h;
      for (int c = 0; c < 2; ++c) {
        for (int q = threadIdx.x; q < W * H; q += kThreads) {
          const int ly = q / W, lx = q - ly * W;
          const int gp = (((y0 + ly) & m) << ln) + ((x0 + lx) & m);
          sb[q] = b[c * np + gp];
          if (!t.first) sw[0][q] = w[c * np + gp];
          if (c == 0) {
            sc[0][q] = cf[gp];
            sc[1][q] = cf[np + gp];
            sc[2][q] = cf[2 * np + gp];
            sc[3][q] = cf[3 * np + gp];
          }
        }
        __syncthreads();
        int src = 0;
        for (int k = 1; k <= h; ++k) {
          const int rw = W - 2 * k, rh = H - 2 * k;
          const double* s0 = sw[src];
          for (int q = threadIdx.x; q < rw * rh; q += kThreads) {
            const int ry = q / rw, rx = q - ry * rw;
            const int wq = (ry + k) * W + rx + k;
            double v;
            if (t.first && k == 1) {
              v = dinv * sb[wq];
            } else {
              double u = sb[wq];
              u = fma(-sc[0][wq], s0[wq + 1], u);
              u = fma(-sc[1][wq], s0[wq - 1], u);
              u = fma(-sc[2][wq], s0[wq + W], u);
              u = fma(-sc[3][wq], s0[wq - W], u);
              v = fma(dinv, u, keep * s0[wq]);
            }
            if (k == h) {
              const int gp = (((y0 + ry + k) & m) << ln) + ((x0 + rx + k) & m);
              wo[c * np + gp] = v;
              if (eo) eo[c * np + gp] = fma(t.c[2], v, eb[c * np + gp]);
            } else {
              sw[src ^ 1][wq] = v;
            }
          }
          __syncthreads();
          src ^= 1;
        }
      }
    } else {
      const int p = threadIdx.x;
      const int i = p & m, j = p >> ln;
      const int pe = (j << ln) + ((i + 1) & m), pw = (j << ln) + ((i - 1) & m);
      const int pn = (((j + 1) & m) << ln) + i, ps = (((j - 1) & m) << ln) + i;
      for (int c = 0; c < 2; ++c) {
        if (p < np) {
          sb[p] = b[c * np + p];
          sw[0][p] = t.first ? 0.0 : w[c * np + p];
          if (c == 0) {
            sc[0][p] = cf[p];
            sc[1][p] = cf[np + p];
            sc[2][p] = cf[2 * np + p];
            sc[3][p] = cf[3 * np + p];
          }
        }
        __syncthreads();
        int src = 0;
        for (int k = 1; k <= h; ++k) {
          if (p < np) {
            const double* s0 = sw[src];
            double v;
            if (t.first && k == 1) {
              v = dinv * sb[p];
            } else {
              double u = sb[p];
              u = fma(-sc[0][p], s0[pe], u);
              u = fma(-sc[1][p], s0[pw], u);
              u = fma(-sc[2][p], s0[pn], u);
              u = fma(-sc[3][p], s0[ps], u);
              v = fma(dinv, u, keep * s0[p]);
            }
            if (k == h) {
              wo[c * np + p] = v;
              if (eo) eo[c * np + p] = fma(t.c[2], v, eb[c * np + p]);
            } else {
              sw[src ^ 1][p] = v;
            }
          }
          __syncthreads();
          src ^= 1;
        }
      }
    }
  });
}

// r = b - A w: in[0] = b, in[1] = w, in[2] = coefficients; c[0] = D.  first:
// the residual after one sweep from zero, which is never stored: w = dinv b
// gives r = (1 - omega) b - dinv sum_k c_k b_k (c[1] = 1 - omega, c[2] = dinv)
__global__ void __launch_bounds__(kThreads) k_mgresid(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const int p = lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    const int np = t.npts;
    const P5 q = nbr(p, t.n, t.logn);
    const double* cf = t.in[2];
    const double ce = cf[p], cw = cf[np + p], cn = cf[2 * np + p], cs = cf[3 * np + p];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double* bc = t.in[0] + c * np;
      double r;
      if (t.first) {
        double sum = ce * bc[q.e];
        sum = fma(cw, bc[q.w], sum);
        sum = fma(cn, bc[q.n], sum);
        sum = fma(cs, bc[q.s], sum);
        r = fma(-t.c[2], sum, t.c[1] * bc[p]);
      } else {
        const double* wc = t.in[1] + c * np;
        double u = bc[p];
        u = fma(-t.c[0], wc[p], u);
        u = fma(-ce, wc[q.e], u);
        u = fma(-cw, wc[q.w], u);
        u = fma(-cn, wc[q.n], u);
        u = fma(-cs, wc[q.s], u);
        r = u;
      }
      t.out[0][c * np + p] = r;
    }
  });
}

// w_f += P w_c (bilinear): one item per coarse point, the four fine points it
// owns; in[0] = coarse correction, out[0] = fine iterate, t.n = fine grid.
// first: w_f = dinv b_f + P w_c (the folded pre-sweep's iterate, never
// stored), with in[1] = b_f and c[0] = dinv
__global__ void __launch_bounds__(kThreads) k_prolong(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const int p = lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    const int nc = t.n >> 1, logc = t.logn - 1, mc = nc - 1, lf = t.logn;
    const int I0 = p & mc, J0 = p >> logc;
    const int I1 = (I0 + 1) & mc, J1 = (J0 + 1) & mc;
    for (int c = 0; c < 2; ++c) {
      const double* g = t.in[0] + (long long)c * t.count;
      double* f = t.out[0] + (long long)c * t.npts;
      const double* bf = t.first ? t.in[1] + (long long)c * t.npts : nullptr;
      const double c00 = g[p], c10 = g[(J0 << logc) + I1];
      const double c01 = g[(J1 << logc) + I0], c11 = g[(J1 << logc) + I1];
      const long long o0 = ((long long)(2 * J0) << lf) + 2 * I0, o1 = o0 + t.n;
      auto base = [&](long long o) { return t.first ? t.c[0] * bf[o] : f[o]; };
      f[o0] = base(o0) + c00;
      f[o0 + 1] = base(o0 + 1) + 0.5 * (c00 + c10);
      f[o1] = base(o1) + 0.5 * (c00 + c01);
      f[o1 + 1] = base(o1 + 1) + 0.25 * ((c00 + c10) + (c01 + c11));
    }
  });
}

// ---------------------------------------------------------------------------
// Block-solve kernels (tasks: block solves)

// z = rhs_blk - sum_{later rows l} R_rl yhat_l (Eq. D+U, mass coupling),
// stored in w; per-chunk ||z||^2; the last chunk starts the FGMRES cycle
__global__ void __launch_bounds__(kThreads) k_fginit(Dev D, int pi) {
  __shared__ double sh[kThreads / 32];
  __shared__ double nrm2[1];
  for_chunks(D, pi, [&](const Task& t, int lc) {
    Sys& S = D.sys[t.sys];
    const Inst& I = D.inst[S.inst];
    const long long q = (long long)lc * kThreads + threadIdx.x;
    double sq = 0.0;
    if (q < t.count) {
      const int rr = (int)(q / I.L);
      const long long p = q - rr * I.L;
      const int r = S.a + rr, s = I.s;
      double z = I.rhs[r * I.L + p];
      for (int l = S.a + S.bs; l < s; ++l) z = fma(-I.R[r * s + l], I.yhat[l * I.L + p], z);
      S.w[q] = z;
      sq = z * z;
    }
    const double tot = cta_sum(sq, sh);
    if (threadIdx.x == 0) D.partials[(long long)(t.pbase + lc) * kPS] = tot;
    if (arrive_last(&S.ctr0, t.nchunk)) {
      reduce_partials(D.partials, t.pbase, t.nchunk, 1, nrm2);
      __syncthreads();
      if (threadIdx.x == 0) {
        S.ctr0 = 0u;
        FGState* f = S.fs;
        const double beta = isfinite(nrm2[0]) ? sqrt(fmax(nrm2[0], 0.0)) : nrm2[0];
        f->j = 0;
        f->k = 0;
        f->its = 0;
        f->guard = 0;
        f->ctr1 = f->ctr2 = 0u;
        f->beta = beta;
        f->target = D.nw[S.inst].eta * beta;
        f->res = beta;
        for (int i = 0; i <= S.m; ++i) f->g[i] = 0.0;
        f->g[0] = beta;
        f->status = isfinite(beta) ? 0 : 2;
        const bool go = beta > 0.0 && isfinite(beta);
        f->stopped = go ? 0 : 1;
        f->inv_scale = go ? 1.0 / beta : 0.0;
      }
    }
  });
}

// block solves whose instance is not iterating stop before they start; the
// Krylov WHILE condition is whether any block solve of the round runs
__global__ void k_kcond(Dev D, int pi, int round, cudaGraphConditionalHandle cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const Plan P = D.plans[pi];
  for (int ti = threadIdx.x; ti < P.ntask; ti += blockDim.x) {
    const Task& t = D.tasks[P.task0 + ti];
    Sys& S = D.sys[t.sys];
    if (!D.nw[S.inst].active) {
      S.fs->stopped = 1;
      S.fs->k = 0;
    }
    if (!S.fs->stopped) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    D.guard[round] = 0;
    cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

// V_0 = z / beta, written to V and to the preconditioner input; yhat_blk = 0
__global__ void __launch_bounds__(kThreads) k_fgscale(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Sys& S = D.sys[t.sys];
    const Inst& I = D.inst[S.inst];
    const long long q = (long long)lc * kThreads + threadIdx.x;
    if (q >= t.count) return;
    const double v = S.w[q] * S.fs->inv_scale;
    S.V[q] = v;
    S.pin[q] = v;
    I.yhat[S.a * I.L + q] = 0.0;
  });
}

// w = D_blk z (Eq. diag_blocks, block-diagonal iteration: the advective part
// on the diagonal terms only) with z = pout; Z_j = z.  One item per point.
// Row r: sum_q R_rq z_q + the advection-diffusion of z_r about Ybar_rr in
// coefficient form (dt nu / h^2 = kd).
__global__ void __launch_bounds__(kThreads) k_matvec(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Sys& S = D.sys[t.sys];
    const Inst& I = D.inst[S.inst];
    const int p = lc * kThreads + threadIdx.x;
    if (p >= t.count) return;
    const int np = I.npts, s = I.s;
    const long long L = I.L;
    const P5 q = nbr(p, I.n, I.logn);
    const double kd = I.dt * I.nu * I.invh2;
    double* Zj = S.Z + (long long)S.fs->j * S.Lb;
    for (int rr = 0; rr < S.bs; ++rr) {
      const int r = S.a + rr;
      const double* xu = S.pout + rr * L;
      const double* xv = xu + np;
      const double* f = I.ccoef + (long long)r * 6 * np + p;
      const double ax = f[0], ay = f[np];
      const double bux = f[2 * np], buy = f[3 * np], bvx = f[4 * np], bvy = f[5 * np];
      const double ce = ax - kd, cw = -ax - kd, cn = ay - kd, cs = -ay - kd;
      const double cc = I.R[r * s + r] + 4.0 * kd;
      const double uc = xu[q.c], vc = xv[q.c];
      double yu = fma(cc + bux, uc, buy * vc);
      yu = fma(ce, xu[q.e], yu);
      yu = fma(cw, xu[q.w], yu);
      yu = fma(cn, xu[q.n], yu);
      yu = fma(cs, xu[q.s], yu);
      double yv = fma(cc + bvy, vc, bvx * uc);
      yv = fma(ce, xv[q.e], yv);
      yv = fma(cw, xv[q.w], yv);
      yv = fma(cn, xv[q.n], yv);
      yv = fma(cs, xv[q.s], yv);
      for (int qq = 0; qq < S.bs; ++qq) {
        if (qq == rr) continue;
        const double m = I.R[r * s + S.a + qq];
        yu = fma(m, S.pout[qq * L + p], yu);
        yv = fma(m, S.pout[qq * L + np + p], yv);
      }
      S.w[rr * L + p] = yu;
      S.w[rr * L + np + p] = yv;
      Zj[rr * L + p] = uc;
      Zj[rr * L + np + p] = vc;
    }
  });
}

// Fused CGS2, as in the single-instance solver: gs1 forms h1 = V^T w; gs2
// updates w -= V h1 and forms h2 = V^T w and ||w||^2, and its last chunk runs
// the Arnoldi/Givens step of the block solve; next forms V_{j+1} = (w - V h2)
// / h_{j+1,j} (the second update is never stored: ||w''||^2 = ||w'||^2 -
// ||h2||^2).  kGsItems items per thread per chunk; partials per chunk and value.
template <int N>
__device__ __forceinline__ void chunk_sums(const double (&vals)[N], int nv, double* sh,
                                           double* dst) {
  // vals[v] (v < nv <= N) of every thread summed over the CTA into dst[v]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < N; ++v) {
    if (v >= nv) break;
    double x = vals[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[v * (kThreads / 32) + wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double r = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) r += sh[threadIdx.x * (kThreads / 32) + k];
    dst[threadIdx.x] = r;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_gs1(Dev D, int pi) {
  __shared__ double sh[kPS * (kThreads / 32)];
  for_chunks(D, pi, [&](const Task& t, int lc) {
    Sys& S = D.sys[t.sys];
    const int nv = S.fs->j + 1;
    const long long q0 = (long long)lc * kGsItems * kThreads + threadIdx.x;
    double wv[kGsItems];
#pragma unroll
    for (int it = 0; it < kGsItems; ++it) {
      const long long q = q0 + (long long)it * kThreads;
      wv[it] = q < t.count ? S.w[q] : 0.0;
    }
    double* dst = D.partials + (long long)(t.pbase + lc) * kPS;
    // four basis vectors at a time: the accumulators stay in registers
    for (int k0 = 0; k0 < nv; k0 += 4) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int it = 0; it < kGsItems; ++it) {
        const long long q = q0 + (long long)it * kThreads;
        if (q >= t.count) break;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          if (k0 + kk < nv) acc[kk] = fma(S.V[(k0 + kk) * S.Lb + q], wv[it], acc[kk]);
      }
      chunk_sums(acc, min(4, nv - k0), sh, dst + k0);
    }
    if (arrive_last(&S.ctr1, t.nchunk)) {
      reduce_partials(D.partials, t.pbase, t.nchunk, nv, S.h1);
      __syncthreads();
      if (threadIdx.x == 0) S.ctr1 = 0u;
    }
  });
}

__device__ void arnoldi(Sys& S, Newton& N, int m) {
  FGState* s = S.fs;
  const int j = s->j, nv = j + 1;
  double* Hc = s->H + j * (IRK_FG_MAXM + 1);
  double h2sq = 0.0;
  for (int i = 0; i <= j; ++i) {
    Hc[i] = S.h1[i] + S.h2[i];
    h2sq = fma(S.h2[i], S.h2[i], h2sq);
  }
  const double rem = S.h2[nv] - h2sq;
  const double hn = rem > 0.0 ? sqrt(rem) : 0.0;
  for (int i = 0; i < j; ++i) {
    const double t0 = s->cs[i] * Hc[i] + s->sn[i] * Hc[i + 1];
    const double t1 = -s->sn[i] * Hc[i] + s->cs[i] * Hc[i + 1];
    Hc[i] = t0;
    Hc[i + 1] = t1;
  }
  const double hjj = Hc[j];
  const double den = hypot(hjj, hn);
  s->cs[j] = den > 0.0 ? hjj / den : 1.0;
  s->sn[j] = den > 0.0 ? hn / den : 0.0;
  Hc[j] = den;
  Hc[j + 1] = 0.0;
  s->g[j + 1] = -s->sn[j] * s->g[j];
  s->g[j] = s->cs[j] * s->g[j];
  const double res = fabs(s->g[j + 1]);
  s->res = res;
  s->its += 1;
  N.kits += 1;
  N.vcyc += S.bs;
  const bool finite = isfinite(hn) && isfinite(res) && isfinite(S.h2[nv]);
  if (!finite) s->status = 2;
  if (!finite || res <= s->target || hn <= 1e-300 || j + 1 >= m) {
    s->k = finite ? j + 1 : 0;
    s->stopped = 1;
  } else {
    s->j = j + 1;
    s->inv_scale = 1.0 / hn;
  }
}

__global__ void __launch_bounds__(kThreads) k_gs2(Dev D, int pi) {
  __shared__ double sh[kPS * (kThreads / 32)];
  for_chunks(D, pi, [&](const Task& t, int lc) {
    Sys& S = D.sys[t.sys];
    const int nv = S.fs->j + 1;
    const long long q0 = (long long)lc * kGsItems * kThreads + threadIdx.x;
    double x[kGsItems];
    double sq = 0.0;
#pragma unroll
    for (int it = 0; it < kGsItems; ++it) {
      const long long q = q0 + (long long)it * kThreads;
      x[it] = 0.0;
      if (q >= t.count) continue;
      double v = S.w[q];
      for (int k = 0; k < nv; ++k) v = fma(-__ldcg(S.h1 + k), S.V[k * S.Lb + q], v);
      S.w[q] = v;
      x[it] = v;
      sq = fma(v, v, sq);
    }
    double* dst = D.partials + (long long)(t.pbase + lc) * kPS;
    for (int k0 = 0; k0 < nv; k0 += 4) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int it = 0; it < kGsItems; ++it) {
        const long long q = q0 + (long long)it * kThreads;
        if (q >= t.count) break;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          if (k0 + kk < nv) acc[kk] = fma(S.V[(k0 + kk) * S.Lb + q], x[it], acc[kk]);
      }
      chunk_sums(acc, min(4, nv - k0), sh, dst + k0);
    }
    const double sqv[1] = {sq};
    chunk_sums(sqv, 1, sh, dst + nv);
    if (arrive_last(&S.ctr2, t.nchunk)) {
      reduce_partials(D.partials, t.pbase, t.nchunk, nv + 1, S.h2);
      __syncthreads();
      __threadfence_block();
      if (threadIdx.x == 0) {
        S.ctr2 = 0u;
        arnoldi(S, D.nw[S.inst], S.m);
      }
    }
  });
}

// V_{j+1} and the next preconditioner input; CTA 0 sets the loop condition
// (any block solve of the round still running) and bounds the loop at m + 1
// body executions independently of the Arnoldi step
__global__ void __launch_bounds__(kThreads) k_next(Dev D, int pi, int round, int limit,
                                                    cudaGraphConditionalHandle cond) {
  if (blockIdx.x == 0) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const Plan P = D.plans[pi];
    const bool over = D.guard[round] + 1 >= limit;
    for (int ti = threadIdx.x; ti < P.ntask; ti += blockDim.x) {
      Sys& S = D.sys[D.tasks[P.task0 + ti].sys];
      if (over && !S.fs->stopped) {
        S.fs->status = 3;
        S.fs->k = S.fs->j + 1;
        S.fs->stopped = 1;
      }
      if (!S.fs->stopped) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      D.guard[round] += 1;
      cudaGraphSetConditional(cond, any ? 1u : 0u);
    }
    __syncthreads();
  }
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Sys& S = D.sys[t.sys];
    const int nv = S.fs->j;  // basis size before the new vector
    const double sc = S.fs->inv_scale;
    double* vn = S.V + (long long)nv * S.Lb;
    for (int it = 0; it < kGsItems; ++it) {
      const long long q = ((long long)lc * kGsItems + it) * kThreads + threadIdx.x;
      if (q >= t.count) break;
      double x = S.w[q];
      for (int v = 0; v < nv; ++v) x = fma(-S.h2[v], S.V[v * S.Lb + q], x);
      x *= sc;
      vn[q] = x;
      S.pin[q] = x;
    }
  });
}

// y = R^{-1} g on the leading k x k triangle, one thread per block solve
__global__ void k_fgsolve(Dev D, int pi) {
  const Plan P = D.plans[pi];
  for (int ti = threadIdx.x; ti < P.ntask; ti += blockDim.x) {
    FGState* s = D.sys[D.tasks[P.task0 + ti].sys].fs;
    if (!D.nw[D.sys[D.tasks[P.task0 + ti].sys].inst].active) continue;
    const int k = s->k;
    for (int i = k - 1; i >= 0; --i) {
      double acc = s->g[i];
      for (int q = i + 1; q < k; ++q) acc -= s->H[q * (IRK_FG_MAXM + 1) + i] * s->y[q];
      s->y[i] = acc / s->H[i * (IRK_FG_MAXM + 1) + i];
    }
  }
}

// yhat_blk = sum_{j<k} y_j Z_j
__global__ void __launch_bounds__(kThreads) k_lincomb(Dev D, int pi) {
  for_chunks(D, pi, [&](const Task& t, int lc) {
    const Sys& S = D.sys[t.sys];
    const Inst& I = D.inst[S.inst];
    const long long q = (long long)lc * kThreads + threadIdx.x;
    if (q >= t.count) return;
    const FGState* f = S.fs;
    double acc = 0.0;
    for (int j = 0; j < f->k; ++j) acc = fma(f->y[j], S.Z[j * S.Lb + q], acc);
    I.yhat[S.a * I.L + q] = acc;
  });
}

// ---------------------------------------------------------------------------
// Host side
enum OpType {
  O_BEGIN, O_F0, O_STATES, O_CCOEF, O_RESID, O_NEWTON, O_REJECT, O_RESTRICT, O_MGCOEF, O_BSWEEP,
  O_MGRESID, O_PROLONG, O_FGINIT, O_KCOND, O_FGSCALE, O_MATVEC, O_GS1, O_GS2, O_NEXT,
  O_FGSOLVE, O_LINCOMB, O_UPDATE, O_FINISH,
  O_NEWTON_BEGIN, O_NEWTON_END, O_KRYLOV_BEGIN, O_KRYLOV_END
};

struct Op {
  int type, plan, mode, round;
  bool operator==(const Op& o) const {
    return type == o.type && plan == o.plan && mode == o.mode && round == o.round;
  }
};

struct RowMG {
  int depth, npre, ncs;
  double sigma, omega, omc;
  double* vel[kMaxLev];   // level 0: the combined field
  double* coef[kMaxLev];
};

struct SysHost {
  int a, bs;
  long long Lb;
  double *V, *Z, *w, *pin, *pout, *tmpb;
  FGState* fs;
  int depth;  // deepest row
  double *mb[kMaxLev], *mw[kMaxLev], *mw2[kMaxLev], *mr[kMaxLev];
};

struct InstHost {
  bool used = false;
  bool own_arena = false;
  irk_config cfg;
  double dt = 0;
  HostTableau tab;
  int n = 0, logn = 0, npts = 0, s = 0, m = 0, nlev = 0;
  long long L = 0;
  void* arena = nullptr;
  size_t bytes = 0;
  Inst d;
  RowMG row[IRK_MAXS];
  SysHost sys[kMaxBlk];
};

struct Layout {
  size_t bytes = 0;
  bool ok = false;
  std::string err;
};

}  // namespace bat
}  // namespace irk

using namespace irk;
using namespace irk::bat;

struct irk_batch {
  int capacity = 0;
  int device = 0;
  cudaStream_t st = nullptr, aux = nullptr, aux2 = nullptr;
  bool own_stream = false;
  std::vector<InstHost> inst;
  std::string err;
  // device tables
  Inst* dinst = nullptr;
  Newton* dnw = nullptr;
  Sys* dsys = nullptr;
  int* dguard = nullptr;
  Plan* dplans = nullptr;
  Task* dtasks = nullptr;
  int* dcs = nullptr;
  double* dpart = nullptr;
  size_t cap_plans = 0, cap_tasks = 0, cap_cs = 0, cap_part = 0;
  // host copies of the program
  std::vector<Plan> plans;
  std::vector<Task> tasks;
  std::vector<int> cs;
  std::vector<int> ctask;
  int* dctask = nullptr;
  size_t cap_ctask = 0;
  int npart = 0;
  std::vector<Op> prog, captured;
  bool dirty = true;
  cudaGraphExec_t exec = nullptr;
  Newton* hnw = nullptr;  // pinned
};

namespace {

const char* set_err(irk_batch* b, const std::string& e) {
  b->err = e;
  return b->err.c_str();
}

#define BCK(x)                                                                  \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      cudaGetLastError();                                                       \
      set_err(b, std::string(#x) + ": " + cudaGetErrorString(e_));              \
      return IRK_ERR_CUDA;                                                      \
    }                                                                           \
  } while (0)

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Depth (levels) of the V-cycle of a row with shift sigma, the depth rule of
// the single-instance solver: stop at the first level where sigma >= D/2
// (D = sigma + 4 dt nu / h_l^2), at least one coarse correction; 0 when no
// level is shift dominated (not accepted here).
int row_depth(int n, double length, int nlev, double sigma, double cdiff) {
  for (int l = 1; l < nlev; ++l) {
    const double hl = length / (n >> l);
    const double D = sigma + 4.0 * cdiff / (hl * hl);
    if (sigma >= 0.5 * D) return l + 1;
  }
  return 0;
}

// Validate cfg and lay out one instance's arena (ih filled when `fill`).
Layout layout(const irk_config* c, double length_check, InstHost* ih, char* base) {
  Layout lo;
  if (!c) { lo.err = "null config"; return lo; }
  if (c->op != IRK_OP_BURGERS_2D) { lo.err = "the batched path serves IRK_OP_BURGERS_2D only"; return lo; }
  if (c->family != IRK_GAUSS && c->family != IRK_RADAU_IIA) { lo.err = "family must be Gauss or Radau IIA"; return lo; }
  if (c->basis != IRK_BASIS_SCHUR) { lo.err = "basis must be the real Schur basis"; return lo; }
  if (c->mg_precision != IRK_MG_FP64) { lo.err = "the batched path runs FP64 V-cycles"; return lo; }
  if (c->nonlinear_variant != 2) { lo.err = "the batched path runs nonlinear_variant 2"; return lo; }
  if (c->forcing) { lo.err = "no forcing on the batched path"; return lo; }
  if (c->mass != IRK_MASS_IDENTITY) { lo.err = "mass must be the identity"; return lo; }
  if (c->n < 32 || c->n > 2048 || (c->n & (c->n - 1))) { lo.err = "n must be a power of two in 32..2048"; return lo; }
  if (c->stages < 1 || c->stages > IRK_MAXS) { lo.err = "stages must be 1..5"; return lo; }
  if (!(c->nu > 0) || !(c->length > 0)) { lo.err = "nu and length must be positive"; return lo; }
  if (c->krylov_restart < 1 || c->krylov_restart > kMaxM) { lo.err = "krylov_restart must be 1..30"; return lo; }
  if (!(c->newton_rtol > 0) || c->newton_maxit < 1 || !(c->krylov_rtol > 0)) { lo.err = "bad Newton/Krylov tolerances"; return lo; }
  (void)length_check;
  HostTableau tab;
  char e[160];
  if (build_tableau(c->family, c->stages, 0, &tab, e, sizeof e) != 0) { lo.err = e; return lo; }
  const int n = c->n, s = c->stages, m = c->krylov_restart;
  int nlev = 0;
  for (int nn = n; nn >= 8; nn >>= 1) ++nlev;
  nlev = std::min(nlev, kMaxLev);
  const long long npts = (long long)n * n, L = 2 * npts;
  // per-row V-cycle depth (the dt of the step enters only through cdiff;
  // validated again with the step's dt in irk_batch_add)
  size_t off = 0;
  auto take = [&](size_t words) -> double* {
    double* p = base ? (double*)(base + off) : nullptr;
    off += ((words * 8 + 255) / 256) * 256;
    return p;
  };
  InstHost tmp;
  InstHost& H = ih ? *ih : tmp;
  H.tab = tab;
  H.n = n;
  H.logn = ilog2(n);
  H.npts = (int)npts;
  H.s = s;
  H.m = m;
  H.nlev = nlev;
  H.L = L;
  H.d.u = take(L);
  H.d.u_save = take(L);
  H.d.K = take(s * L);
  H.d.Y = take(s * L);
  H.d.combos = take(s * L);
  H.d.ccoef = take((size_t)s * 6 * npts);
  H.d.rhs = take(s * L);
  H.d.yhat = take(s * L);
  // rows: velocity (levels >= 1) and coefficients of every level the row may
  // reach (allocated for the whole hierarchy; the depth depends on dt)
  for (int r = 0; r < s; ++r) {
    RowMG& R = H.row[r];
    for (int l = 0; l < nlev; ++l) {
      const long long nl = (long long)(n >> l) * (n >> l);
      R.vel[l] = l == 0 ? nullptr : take(2 * nl);
      R.coef[l] = take(4 * nl);
    }
  }
  // The block solves of one instance run one after another (back
  // substitution), so they share one set of Krylov and multigrid work
  // buffers, sized for the largest block; each keeps its own FGMRES state.
  int bsmax = 1;
  for (int k = 0; k < tab.nblk; ++k) bsmax = std::max(bsmax, tab.bsize[k]);
  const long long Lmax = bsmax * L;
  double* V = take((m + 1) * Lmax);
  double* Z = take(m * Lmax);
  double* w = take(Lmax);
  double* pin = take(Lmax);
  double* pout = take(Lmax);
  double* tmpb = take(L);
  double *mb[kMaxLev], *mw[kMaxLev], *mw2[kMaxLev], *mr[kMaxLev];
  for (int l = 0; l < nlev; ++l) {
    const long long nl = (long long)(n >> l) * (n >> l);
    mb[l] = l == 0 ? nullptr : take(2 * nl);
    mw[l] = take(2 * nl);
    mw2[l] = take(2 * nl);
    mr[l] = take(2 * nl);
  }
  for (int k = 0; k < tab.nblk; ++k) {
    SysHost& S = H.sys[k];
    S.a = tab.bstart[k];
    S.bs = tab.bsize[k];
    S.Lb = S.bs * L;
    S.V = V;
    S.Z = Z;
    S.w = w;
    S.pin = pin;
    S.pout = pout;
    S.tmpb = tmpb;
    S.fs = (FGState*)take((sizeof(FGState) + 7) / 8);
    for (int l = 0; l < nlev; ++l) {
      S.mb[l] = mb[l];
      S.mw[l] = mw[l];
      S.mw2[l] = mw2[l];
      S.mr[l] = mr[l];
    }
  }
  lo.bytes = off;
  lo.ok = true;
  return lo;
}

// Fill the per-row multigrid data for the step dt; false (with err) if a
// row's V-cycle is not shift dominated on its coarsest level.
bool setup_rows(InstHost& H, double dt, std::string& err) {
  const double cdiff = dt * H.cfg.nu;
  const double om = H.cfg.mg_omega > 0 ? H.cfg.mg_omega : 0.8;
  const double red = H.cfg.mg_coarse_reduction > 0 ? H.cfg.mg_coarse_reduction : 2e-2;
  for (int r = 0; r < H.s; ++r) {
    RowMG& R = H.row[r];
    int blk = 0;
    for (int k = 0; k < H.tab.nblk; ++k)
      if (r >= H.tab.bstart[k] && r < H.tab.bstart[k] + H.tab.bsize[k]) blk = k;
    const bool first = (r == H.tab.bstart[blk]);
    R.sigma = first ? H.tab.eta[blk] : (H.cfg.gamma_mode == 1 ? H.tab.eta[blk] : H.tab.gamma_star[blk]);
    R.depth = row_depth(H.n, H.cfg.length, H.nlev, R.sigma, cdiff);
    R.omega = om;
    if (R.depth == 0) {
      err = "a V-cycle row is not shift dominated on any level (dt nu too large for the "
            "batched path)";
      return false;
    }
    const double h0 = H.cfg.length / H.n;
    const double D0 = R.sigma + 4.0 * cdiff / (h0 * h0);
    R.npre = (H.cfg.mg_shifted_sweeps > 0 && R.sigma >= 0.15 * D0) ? H.cfg.mg_shifted_sweeps
                                                                   : std::max(1, H.cfg.mg_pre);
    const double hc = H.cfg.length / (H.n >> (R.depth - 1));
    const double D = R.sigma + 4.0 * cdiff / (hc * hc);
    R.omc = (R.sigma >= 0.5 * D) ? 1.0 : om;
    const double rho = 1.0 - R.omc * R.sigma / D;
    int sw = (rho > 0 && rho < 1) ? (int)std::ceil(std::log(red) / std::log(rho)) : 2;
    R.ncs = std::max(2, std::min(sw, 12));
    R.vel[0] = H.d.combos + (long long)r * H.L;
  }
  for (int k = 0; k < H.tab.nblk; ++k) {
    SysHost& S = H.sys[k];
    S.depth = 0;
    for (int rr = 0; rr < S.bs; ++rr) S.depth = std::max(S.depth, H.row[S.a + rr].depth);
  }
  return true;
}

// ---- program construction --------------------------------------------------
// The device word a task's flag tests, and the sense of the test.
void set_flag(irk_batch* b, Task& t) {
  t.flagp = nullptr;
  t.on_nonzero = 1;
  switch (t.flag) {
    case F_INST:
      t.flagp = &b->dnw[t.inst].active;
      break;
    case F_REJ:
      t.flagp = &b->dnw[t.inst].rejected;
      break;
    case F_SYS:
      t.flagp = &b->inst[t.sys / kMaxBlk].sys[t.sys % kMaxBlk].fs->stopped;
      t.on_nonzero = 0;
      break;
    default:
      break;
  }
}

struct Builder {
  irk_batch* b;
  int addplan(const std::vector<Task>& ts, int ipc, bool reduce) {
    Plan P;
    P.ntask = (int)ts.size();
    P.task0 = (int)b->tasks.size();
    P.cs0 = (int)b->cs.size();
    int c = 0;
    for (Task t : ts) {
      t.nchunk = (t.count + ipc - 1) / ipc;
      if (reduce) {
        t.pbase = b->npart;
        b->npart += t.nchunk;
      }
      set_flag(b, t);
      b->cs.push_back(c);
      c += t.nchunk;
      b->tasks.push_back(t);
    }
    b->cs.push_back(c);
    P.nchunk = c;
    b->plans.push_back(P);
    // task of chunk k for CTA k (chunks of a task are consecutive)
    int ti = 0;
    for (int k = 0; k < kGrid; ++k) {
      if (k >= c) {
        b->ctask.push_back(0);
        continue;
      }
      while (b->cs[P.cs0 + ti + 1] <= k) ++ti;
      b->ctask.push_back(ti);
    }
    return (int)b->plans.size() - 1;
  }
  void op(int type, int plan, int mode = 0, int round = 0) { b->prog.push_back({type, plan, mode, round}); }
};

Task inst_task(const InstHost& H, int slot, long long count, int flag) {
  Task t;
  memset(&t, 0, sizeof(t));
  t.n = H.n;
  t.logn = H.logn;
  t.npts = H.npts;
  t.count = (int)count;
  t.inst = slot;
  t.sys = -1;
  t.flag = flag;
  return t;
}

Task lev_task(const InstHost& H, int slot, int sysi, int l, long long count, int flag) {
  Task t;
  memset(&t, 0, sizeof(t));
  t.n = H.n >> l;
  t.logn = H.logn - l;
  t.npts = t.n * t.n;
  t.count = (int)count;
  t.inst = slot;
  t.sys = sysi;
  t.flag = flag;
  return t;
}

// MG constants of row R on level l: D, omega/D, 1 - omega
void mg_consts(const InstHost& H, const RowMG& R, int l, double omega, double* D, double* dinv,
               double* keep) {
  const double hl = H.cfg.length / (H.n >> l);
  *D = R.sigma + 4.0 * H.dt * H.cfg.nu / (hl * hl);
  *dinv = omega / *D;
  *keep = 1.0 - omega;
}

// One V-cycle phase: the rows `rows` (instance slot, block index, row in
// block), each from its level-0 input to its output, in lock step.  On level
// l a row going deeper takes its pre-sweeps (a single pre-sweep from zero is
// folded into the residual and the prolongation, as in the single-instance
// solver) and a row whose coarsest level is l takes its coarse sweeps, both
// in the same k_bsweep launches of up to three sweeps each.  epi_out: the
// pointwise L_P coupling row written by the row's last sweep.
struct PhaseRow {
  int slot, blk, rr;
  const double* in;
  double* out;
  double* epi_out;
  const double* epi_base;
  double epi_coef;
};

void emit_vcycle(irk_batch* b, Builder& B, const std::vector<PhaseRow>& rows) {
  if (rows.empty()) return;
  const size_t nr = rows.size();
  auto Rof = [&](size_t i) -> RowMG& {
    InstHost& H = b->inst[rows[i].slot];
    return H.row[H.sys[rows[i].blk].a + rows[i].rr];
  };
  auto Hof = [&](size_t i) -> InstHost& { return b->inst[rows[i].slot]; };
  auto Sof = [&](size_t i) -> SysHost& { return b->inst[rows[i].slot].sys[rows[i].blk]; };
  auto sysi = [&](size_t i) { return rows[i].slot * kMaxBlk + rows[i].blk; };
  auto bl = [&](size_t i, int l) -> const double* { return l == 0 ? rows[i].in : Sof(i).mb[l]; };
  int Dmax = 0;
  for (size_t i = 0; i < nr; ++i) Dmax = std::max(Dmax, Rof(i).depth);
  std::vector<const double*> cur(nr * kMaxLev, nullptr);
  std::vector<int> which(nr * kMaxLev, 0);
  auto nextbuf = [&](size_t i, int l) -> double* {
    SysHost& S = Sof(i);
    double* o = which[i * kMaxLev + l] == 0 ? S.mw[l] : S.mw2[l];
    which[i * kMaxLev + l] ^= 1;
    return o;
  };
  auto folded = [&](size_t i) { return Rof(i).npre == 1; };
  auto points = [&](size_t i, int l) { return (long long)(Hof(i).n >> l) * (Hof(i).n >> l); };
  auto tiles = [&](size_t i, int l) {
    const int nl = Hof(i).n >> l;
    return nl >= kBX ? (long long)(nl / kBX) * (nl / kBY) : 1LL;
  };
  // sweeps of row i on level l on the way down
  auto down_sweeps = [&](size_t i, int l) {
    const RowMG& R = Rof(i);
    if (R.depth - 1 > l) return folded(i) ? 0 : R.npre;
    if (R.depth - 1 == l) return R.ncs;
    return 0;
  };
  auto sweep_task = [&](size_t i, int l, int nsw, bool first, double omega, double* out,
                        bool epi) {
    InstHost& H = Hof(i);
    RowMG& R = Rof(i);
    Task t = lev_task(H, rows[i].slot, sysi(i), l, tiles(i, l), F_SYS);
    double Dg, dinv, keep;
    mg_consts(H, R, l, omega, &Dg, &dinv, &keep);
    t.c[0] = dinv;
    t.c[1] = keep;
    t.first = first;
    t.nsw = nsw;
    t.in[0] = bl(i, l);
    t.in[1] = cur[i * kMaxLev + l];
    t.in[2] = R.coef[l];
    t.out[0] = out;
    if (epi && rows[i].epi_out) {
      t.out[1] = rows[i].epi_out;
      t.in[3] = rows[i].epi_base;
      t.c[2] = rows[i].epi_coef;
    }
    return t;
  };
  for (int l = 0; l < Dmax; ++l) {
    int nlaunch = 0;
    for (size_t i = 0; i < nr; ++i) nlaunch = std::max(nlaunch, (down_sweeps(i, l) + 2) / 3);
    for (int k = 0; k < nlaunch; ++k) {
      std::vector<Task> ts;
      for (size_t i = 0; i < nr; ++i) {
        const int S = down_sweeps(i, l);
        if (3 * k >= S) continue;
        const RowMG& R = Rof(i);
        const double om = (R.depth - 1 == l) ? R.omc : R.omega;
        double* o = nextbuf(i, l);
        ts.push_back(sweep_task(i, l, std::min(3, S - 3 * k), k == 0, om, o, false));
        cur[i * kMaxLev + l] = o;
      }
      B.op(O_BSWEEP, B.addplan(ts, 1, false));
    }
    std::vector<Task> tr, trs;
    for (size_t i = 0; i < nr; ++i) {
      RowMG& R = Rof(i);
      if (R.depth - 1 <= l) continue;
      InstHost& H = Hof(i);
      SysHost& S = Sof(i);
      Task t = lev_task(H, rows[i].slot, sysi(i), l, points(i, l), F_SYS);
      double Dg, dinv, keep;
      mg_consts(H, R, l, R.omega, &Dg, &dinv, &keep);
      t.c[0] = Dg;
      t.c[1] = keep;
      t.c[2] = dinv;
      t.first = folded(i);
      t.in[0] = bl(i, l);
      t.in[1] = cur[i * kMaxLev + l];
      t.in[2] = R.coef[l];
      t.out[0] = S.mr[l];
      tr.push_back(t);
      Task u = lev_task(H, rows[i].slot, sysi(i), l, points(i, l + 1), F_SYS);
      u.in[0] = S.mr[l];
      u.out[0] = S.mb[l + 1];
      trs.push_back(u);
    }
    if (!tr.empty()) {
      B.op(O_MGRESID, B.addplan(tr, kThreads, false));
      B.op(O_RESTRICT, B.addplan(trs, kThreads, false));
    }
  }
  for (int l = Dmax - 2; l >= 0; --l) {
    std::vector<Task> tp;
    int nlaunch = 0;
    for (size_t i = 0; i < nr; ++i) {
      RowMG& R = Rof(i);
      if (R.depth - 1 <= l) continue;
      InstHost& H = Hof(i);
      Task t = lev_task(H, rows[i].slot, sysi(i), l, points(i, l + 1), F_SYS);
      t.in[0] = cur[i * kMaxLev + l + 1];
      if (folded(i)) {
        double Dg, dinv, keep;
        mg_consts(H, R, l, R.omega, &Dg, &dinv, &keep);
        t.first = 1;
        t.c[0] = dinv;
        t.in[1] = bl(i, l);
        double* o = nextbuf(i, l);
        t.out[0] = o;
        cur[i * kMaxLev + l] = o;
      } else {
        t.out[0] = const_cast<double*>(cur[i * kMaxLev + l]);
      }
      tp.push_back(t);
      nlaunch = std::max(nlaunch, (R.npre + 2) / 3);
    }
    if (tp.empty()) continue;
    B.op(O_PROLONG, B.addplan(tp, kThreads, false));
    for (int k = 0; k < nlaunch; ++k) {
      std::vector<Task> ts;
      for (size_t i = 0; i < nr; ++i) {
        RowMG& R = Rof(i);
        if (R.depth - 1 <= l || 3 * k >= R.npre) continue;
        const int nsw = std::min(3, R.npre - 3 * k);
        const bool last = (3 * k + nsw == R.npre);
        double* o = (l == 0 && last) ? rows[i].out : nextbuf(i, l);
        ts.push_back(sweep_task(i, l, nsw, false, R.omega, o, l == 0 && last));
        cur[i * kMaxLev + l] = o;
      }
      B.op(O_BSWEEP, B.addplan(ts, 1, false));
    }
  }
}

// Build the whole step program for the resident instances.
void build_program(irk_batch* b) {
  b->plans.clear();
  b->tasks.clear();
  b->cs.clear();
  b->ctask.clear();
  b->prog.clear();
  b->npart = 0;
  Builder B{b};
  std::vector<int> slots;
  for (int k = 0; k < b->capacity; ++k)
    if (b->inst[k].used) slots.push_back(k);
  auto per_inst = [&](long long (*cnt)(const InstHost&), int flag, bool reduce) {
    std::vector<Task> ts;
    for (int k : slots) ts.push_back(inst_task(b->inst[k], k, cnt(b->inst[k]), flag));
    return B.addplan(ts, kThreads, reduce);
  };
  auto cL = [](const InstHost& H) { return H.L; };
  auto c2 = [](const InstHost& H) { return 2LL * H.npts; };
  auto c1 = [](const InstHost& H) { return (long long)H.npts; };
  auto cK = [](const InstHost& H) { return H.s * H.L; };
  // ---- prefix
  {
    std::vector<Task> ts;
    for (int k : slots) {
      Task t = inst_task(b->inst[k], k, b->inst[k].L, F_NONE);
      t.c[0] = 1.0;  // extrapolate the previous stages (zero after add or a failure)
      ts.push_back(t);
    }
    B.op(O_BEGIN, B.addplan(ts, kThreads, false));
  }
  const int pf0 = per_inst(c2, F_NONE, true);
  B.op(O_F0, pf0);
  B.op(O_STATES, per_inst(cL, F_NONE, false));
  B.op(O_CCOEF, per_inst(c1, F_NONE, false));
  const int pr0 = per_inst(c2, F_NONE, true);
  B.op(O_RESID, pr0);
  auto newton_plan = [&](int presid) {
    std::vector<Task> ts;
    const Plan& R = b->plans[presid];
    const Plan& F = b->plans[pf0];
    for (int i = 0; i < (int)slots.size(); ++i) {
      Task t = b->tasks[R.task0 + i];
      t.p2base = b->tasks[F.task0 + i].pbase;
      t.n2chunk = b->tasks[F.task0 + i].nchunk;
      ts.push_back(t);
    }
    // keep the residual's partial ranges: add without new partials
    Plan P;
    P.ntask = (int)ts.size();
    P.task0 = (int)b->tasks.size();
    P.cs0 = (int)b->cs.size();
    P.nchunk = 0;
    for (auto& t : ts) {
      b->tasks.push_back(t);
      b->cs.push_back(0);
    }
    b->cs.push_back(0);
    b->plans.push_back(P);
    for (int k = 0; k < kGrid; ++k) b->ctask.push_back(0);
    return (int)b->plans.size() - 1;
  };
  B.op(O_NEWTON, newton_plan(pr0), N_FIRST);
  B.op(O_REJECT, per_inst(cK, F_REJ, false));
  B.op(O_STATES, per_inst(cL, F_REJ, false));
  B.op(O_CCOEF, per_inst(c1, F_REJ, false));
  const int pr1 = per_inst(c2, F_REJ, true);
  B.op(O_RESID, pr1);
  B.op(O_NEWTON, newton_plan(pr1), N_RECHECK);
  // ---- Newton loop
  B.op(O_NEWTON_BEGIN, -1);
  {
    // multigrid coefficient hierarchy of every row of the iterating instances
    int Dmax = 0;
    for (int k : slots)
      for (int r = 0; r < b->inst[k].s; ++r) Dmax = std::max(Dmax, b->inst[k].row[r].depth);
    for (int l = 0; l + 1 < Dmax; ++l) {
      std::vector<Task> ts;
      for (int k : slots) {
        InstHost& H = b->inst[k];
        for (int r = 0; r < H.s; ++r) {
          if (H.row[r].depth - 1 <= l) continue;
          Task t = lev_task(H, k, -1, l, (long long)(H.n >> (l + 1)) * (H.n >> (l + 1)), F_INST);
          t.in[0] = H.row[r].vel[l];
          t.out[0] = H.row[r].vel[l + 1];
          ts.push_back(t);
        }
      }
      if (!ts.empty()) B.op(O_RESTRICT, B.addplan(ts, kThreads, false));
    }
    std::vector<Task> tc;
    for (int k : slots) {
      InstHost& H = b->inst[k];
      for (int r = 0; r < H.s; ++r)
        for (int l = 0; l < H.row[r].depth; ++l) {
          Task t = lev_task(H, k, -1, l, (long long)(H.n >> l) * (H.n >> l), F_INST);
          const double hl = H.cfg.length / (H.n >> l);
          t.c[0] = H.dt / (2.0 * hl);
          t.c[1] = -H.dt * H.cfg.nu / (hl * hl);
          t.in[0] = H.row[r].vel[l];
          t.out[0] = H.row[r].coef[l];
          tc.push_back(t);
        }
    }
    B.op(O_MGCOEF, B.addplan(tc, kThreads, false));
    // block solves, from the last Schur block of every instance
    int rounds = 0;
    for (int k : slots) rounds = std::max(rounds, b->inst[k].tab.nblk);
    for (int rd = 0; rd < rounds; ++rd) {
      std::vector<Task> sysT, sysG;
      std::vector<PhaseRow> ra, rb;
      for (int k : slots) {
        InstHost& H = b->inst[k];
        const int blk = H.tab.nblk - 1 - rd;
        if (blk < 0) continue;
        SysHost& S = H.sys[blk];
        const int sysi = k * kMaxBlk + blk;
        Task t = inst_task(H, k, S.Lb, F_SYS);
        t.sys = sysi;
        sysT.push_back(t);
        Task g = t;
        sysG.push_back(g);
        if (S.bs == 2) {
          // r_b' = v_b - R_ba z_a, written by the last sweep of row a's V-cycle
          ra.push_back({k, blk, 0, S.pin, S.pout, S.tmpb, S.pin + H.L,
                        -H.tab.R[(S.a + 1) * H.s + S.a]});
          rb.push_back({k, blk, 1, S.tmpb, S.pout + H.L, nullptr, nullptr, 0.0});
        } else {
          ra.push_back({k, blk, 0, S.pin, S.pout, nullptr, nullptr, 0.0});
        }
      }
      std::vector<Task> sysInit = sysT;
      for (auto& t : sysInit) t.flag = F_INST;
      const int pinit = B.addplan(sysInit, kThreads, true);
      B.op(O_FGINIT, pinit);
      B.op(O_KCOND, pinit, 0, rd);
      B.op(O_FGSCALE, B.addplan(sysT, kThreads, false));
      B.op(O_KRYLOV_BEGIN, -1, 0, rd);
      emit_vcycle(b, B, ra);
      emit_vcycle(b, B, rb);
      std::vector<Task> mv;
      for (auto& t : sysT) {
        Task u = t;
        u.count = b->inst[t.inst].npts;
        mv.push_back(u);
      }
      B.op(O_MATVEC, B.addplan(mv, kThreads, false));
      B.op(O_GS1, B.addplan(sysG, kThreads * kGsItems, true));
      B.op(O_GS2, B.addplan(sysG, kThreads * kGsItems, true));
      B.op(O_NEXT, B.addplan(sysG, kThreads * kGsItems, false), 0, rd);
      B.op(O_KRYLOV_END, -1, 0, rd);
      B.op(O_FGSOLVE, pinit);
      std::vector<Task> lc = sysT;
      for (auto& t : lc) t.flag = F_INST;
      B.op(O_LINCOMB, B.addplan(lc, kThreads, false));
    }
    B.op(O_UPDATE, per_inst(cL, F_INST, false));
    B.op(O_STATES, per_inst(cL, F_INST, false));
    B.op(O_CCOEF, per_inst(c1, F_INST, false));
    const int pr2 = per_inst(c2, F_INST, true);
    B.op(O_RESID, pr2);
    B.op(O_NEWTON, newton_plan(pr2), N_CTL);
  }
  B.op(O_NEWTON_END, -1);
  B.op(O_FINISH, per_inst(cL, F_NONE, false));
}

irk_status upload(irk_batch* b, bool* realloc_done) {
  *realloc_done = false;
  auto grow = [&](void** p, size_t* cap, size_t need) -> cudaError_t {
    if (need <= *cap) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    const size_t n = need + need / 2 + 1024;
    cudaError_t e = cudaMalloc(p, n);
    *cap = e == cudaSuccess ? n : 0;
    *realloc_done = true;
    return e;
  };
  BCK(grow((void**)&b->dplans, &b->cap_plans, b->plans.size() * sizeof(Plan)));
  BCK(grow((void**)&b->dtasks, &b->cap_tasks, b->tasks.size() * sizeof(Task)));
  BCK(grow((void**)&b->dcs, &b->cap_cs, b->cs.size() * sizeof(int)));
  BCK(grow((void**)&b->dctask, &b->cap_ctask, b->ctask.size() * sizeof(int)));
  BCK(grow((void**)&b->dpart, &b->cap_part, (size_t)std::max(b->npart, 1) * kPS * sizeof(double)));
  BCK(cudaMemcpyAsync(b->dplans, b->plans.data(), b->plans.size() * sizeof(Plan),
                      cudaMemcpyHostToDevice, b->st));
  BCK(cudaMemcpyAsync(b->dtasks, b->tasks.data(), b->tasks.size() * sizeof(Task),
                      cudaMemcpyHostToDevice, b->st));
  BCK(cudaMemcpyAsync(b->dcs, b->cs.data(), b->cs.size() * sizeof(int), cudaMemcpyHostToDevice,
                      b->st));
  BCK(cudaMemcpyAsync(b->dctask, b->ctask.data(), b->ctask.size() * sizeof(int),
                      cudaMemcpyHostToDevice, b->st));
  BCK(cudaStreamSynchronize(b->st));  // the host vectors may change before the next step
  return IRK_OK;
}

// Capture the program into one graph (conditional WHILE nodes for the loops).
irk_status capture(irk_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  Dev D;
  D.plans = b->dplans;
  D.tasks = b->dtasks;
  D.cs = b->dcs;
  D.ctask = b->dctask;
  D.inst = b->dinst;
  D.nw = b->dnw;
  D.sys = b->dsys;
  D.partials = b->dpart;
  D.guard = b->dguard;
  cudaGraph_t G = nullptr;
  BCK(cudaGraphCreate(&G, 0));
  cudaGraphConditionalHandle ncond = 0;
  cudaError_t e = cudaGraphConditionalHandleCreate(&ncond, G, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(b->st, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  cudaStream_t cur = b->st;
  cudaGraph_t nbody_graph = nullptr;
  cudaGraphConditionalHandle kcond[kMaxBlk] = {0, 0, 0};
  cudaGraphNode_t wnode = nullptr, kwnode = nullptr;
  auto add_while = [&](cudaStream_t s, cudaGraph_t g, cudaGraphConditionalHandle h,
                       cudaGraphNode_t* node, cudaGraph_t* body) -> cudaError_t {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t r = cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (r != cudaSuccess) return r;
    if (cst != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    r = cudaGraphAddNode(node, g, deps, nullptr, ndeps, &np);
    if (r == cudaSuccess) *body = np.conditional.phGraph_out[0];
    return r;
  };
  for (size_t i = 0; i < b->prog.size() && e == cudaSuccess; ++i) {
    const Op& o = b->prog[i];
    const int pi = o.plan;
    switch (o.type) {
      case O_BEGIN: k_begin<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_F0: k_f0<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_STATES: k_states<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_CCOEF: k_ccoef<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_RESID: k_resid<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_NEWTON: k_newton<<<1, 256, 0, cur>>>(D, pi, o.mode, ncond); break;
      case O_REJECT: k_reject<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_RESTRICT: k_restrict<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_MGCOEF: k_mgcoef<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_BSWEEP: k_bsweep<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_MGRESID: k_mgresid<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_PROLONG: k_prolong<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_FGINIT: k_fginit<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_KCOND: k_kcond<<<1, 256, 0, cur>>>(D, pi, o.round, kcond[o.round]); break;
      case O_FGSCALE: k_fgscale<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_MATVEC: k_matvec<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_GS1: k_gs1<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_GS2: k_gs2<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_NEXT: k_next<<<kGrid, kThreads, 0, cur>>>(D, pi, o.round, kMaxM + 1, kcond[o.round]); break;
      case O_FGSOLVE: k_fgsolve<<<1, 256, 0, cur>>>(D, pi); break;
      case O_LINCOMB: k_lincomb<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_UPDATE: k_update<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_FINISH: k_finish<<<kGrid, kThreads, 0, cur>>>(D, pi); break;
      case O_NEWTON_BEGIN: {
        e = add_while(b->st, G, ncond, &wnode, &nbody_graph);
        if (e == cudaSuccess)
          e = cudaStreamBeginCaptureToGraph(b->aux, nbody_graph, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        // the Krylov conditions live in the Newton body graph (one per round)
        int nround = 0;
        for (const Op& q : b->prog) nround += (q.type == O_KRYLOV_BEGIN) ? 1 : 0;
        for (int r = 0; r < nround && e == cudaSuccess; ++r)
          e = cudaGraphConditionalHandleCreate(&kcond[r], nbody_graph, 1, cudaGraphCondAssignDefault);
        cur = b->aux;
        break;
      }
      case O_NEWTON_END: {
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(b->aux, &out);
        if (e == cudaSuccess)
          e = cudaStreamUpdateCaptureDependencies(b->st, &wnode, nullptr, 1,
                                                  cudaStreamSetCaptureDependencies);
        cur = b->st;
        break;
      }
      case O_KRYLOV_BEGIN: {
        cudaGraph_t kbody = nullptr;
        e = add_while(b->aux, nbody_graph, kcond[o.round], &kwnode, &kbody);
        if (e == cudaSuccess)
          e = cudaStreamBeginCaptureToGraph(b->aux2, kbody, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        cur = b->aux2;
        break;
      }
      case O_KRYLOV_END: {
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(b->aux2, &out);
        if (e == cudaSuccess)
          e = cudaStreamUpdateCaptureDependencies(b->aux, &kwnode, nullptr, 1,
                                                  cudaStreamSetCaptureDependencies);
        cur = b->aux;
        break;
      }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->st, &out);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, G, 0);
  cudaGraphDestroy(G);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->exec = nullptr;
    set_err(b, std::string("graph capture failed: ") + cudaGetErrorString(e));
    return IRK_ERR_CUDA;
  }
  b->captured = b->prog;
  return IRK_OK;
}

// Device descriptors of slot k (instance, block solves).
irk_status write_slot(irk_batch* b, int k) {
  InstHost& H = b->inst[k];
  Inst& d = H.d;
  d.s = H.s;
  d.n = H.n;
  d.logn = H.logn;
  d.npts = H.npts;
  d.L = H.L;
  d.dt = H.dt;
  d.nu = H.cfg.nu;
  d.h = H.cfg.length / H.n;
  d.inv2h = 0.5 / d.h;
  d.invh2 = 1.0 / (d.h * d.h);
  d.newton_rtol = H.cfg.newton_rtol;
  d.krylov_rtol = H.cfg.krylov_rtol;
  d.newton_maxit = H.cfg.newton_maxit;
  const int s = H.s;
  for (int i = 0; i < s * s; ++i) {
    d.A[i] = H.tab.A[i];
    d.TR[i] = H.tab.TR[i];
    d.R[i] = H.tab.R[i];
    d.Tinv[i] = H.tab.Tinv[i];
  }
  for (int i = 0; i < s; ++i) d.b[i] = H.tab.b[i];
  // diagonal combined fields: Ybar_kk = sum_m (T^{-1})_km T_mk Y_m
  for (int k2 = 0; k2 < s; ++k2)
    for (int m = 0; m < s; ++m) d.Dd[k2 * s + m] = H.tab.Tinv[k2 * s + m] * H.tab.T[m * s + k2];
  // Newton start: the previous stages extrapolated along the collocation
  // polynomial to this step's nodes (same dt: ratio 1), k_j = sum_i k_i l_i(1 + c_j)
  for (int j = 0; j < s; ++j)
    for (int i = 0; i < s; ++i) {
      long double l = 1.0L;
      const long double th = 1.0L + (long double)H.tab.c[j];
      for (int m = 0; m < s; ++m)
        if (m != i) l *= (th - H.tab.c[m]) / ((long double)H.tab.c[i] - H.tab.c[m]);
      d.E[j * s + i] = (s > 1) ? (double)l : 1.0;
    }
  BCK(cudaMemcpyAsync(b->dinst + k, &d, sizeof(Inst), cudaMemcpyHostToDevice, b->st));
  for (int q = 0; q < H.tab.nblk; ++q) {
    SysHost& S = H.sys[q];
    Sys ds;
    memset(&ds, 0, sizeof(ds));
    ds.inst = k;
    ds.a = S.a;
    ds.bs = S.bs;
    ds.m = H.m;
    ds.Lb = S.Lb;
    ds.V = S.V;
    ds.Z = S.Z;
    ds.w = S.w;
    ds.pin = S.pin;
    ds.pout = S.pout;
    ds.tmpb = S.tmpb;
    ds.fs = S.fs;
    BCK(cudaMemcpyAsync(b->dsys + k * kMaxBlk + q, &ds, sizeof(Sys), cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemsetAsync(S.fs, 0, sizeof(FGState), b->st));
  }
  return IRK_OK;
}

}  // namespace

extern "C" {

irk_status irk_batch_create(int capacity, void* cuda_stream, irk_batch** out) {
  if (!out || capacity < 1 || capacity > 64) return IRK_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return IRK_ERR_NO_DEVICE;
  }
  irk_batch* b = new irk_batch();
  b->capacity = capacity;
  cudaGetDevice(&b->device);
  b->inst.resize(capacity);
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->st = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->aux2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->dinst, sizeof(Inst) * capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->dnw, sizeof(Newton) * capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->dsys, sizeof(Sys) * capacity * kMaxBlk);
  if (e == cudaSuccess) e = cudaMalloc(&b->dguard, sizeof(int) * kMaxBlk);
  if (e == cudaSuccess) e = cudaMallocHost(&b->hnw, sizeof(Newton) * capacity);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dnw, 0, sizeof(Newton) * capacity, b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dsys, 0, sizeof(Sys) * capacity * kMaxBlk, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    irk_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? IRK_ERR_NOMEM : IRK_ERR_CUDA;
  }
  *out = b;
  return IRK_OK;
}

size_t irk_batch_instance_bytes(const irk_config* cfg) {
  Layout lo = layout(cfg, 0, nullptr, nullptr);
  return lo.ok ? lo.bytes : 0;
}

irk_status irk_batch_add(irk_batch* b, const irk_config* cfg, const double* u0, int u0_on_device,
                         double dt, void* arena, size_t arena_bytes, int* slot) {
  if (!b) return IRK_ERR_INVALID;
  DeviceScope ds(b->device);
  if (!cfg || !u0 || !slot || !(dt > 0) || !std::isfinite(dt)) {
    set_err(b, "cfg, u0, slot and dt > 0 are required");
    return IRK_ERR_INVALID;
  }
  Layout lo = layout(cfg, 0, nullptr, nullptr);
  if (!lo.ok) {
    set_err(b, lo.err);
    return IRK_ERR_INVALID;
  }
  int k = -1;
  for (int i = 0; i < b->capacity && k < 0; ++i)
    if (!b->inst[i].used) k = i;
  if (k < 0) {
    set_err(b, "the batch is full");
    return IRK_ERR_NOMEM;
  }
  InstHost& H = b->inst[k];
  H = InstHost();
  H.cfg = *cfg;
  H.dt = dt;
  if (arena) {
    if (arena_bytes < lo.bytes || ((uintptr_t)arena & 255)) {
      set_err(b, "arena too small or not 256-byte aligned");
      return IRK_ERR_INVALID;
    }
    H.arena = arena;
  } else {
    if (cudaMalloc(&H.arena, lo.bytes) != cudaSuccess) {
      cudaGetLastError();
      set_err(b, "cudaMalloc of the instance arena failed");
      return IRK_ERR_NOMEM;
    }
    H.own_arena = true;
  }
  H.bytes = lo.bytes;
  layout(cfg, 0, &H, (char*)H.arena);
  std::string err;
  if (!setup_rows(H, dt, err)) {
    if (H.own_arena) cudaFree(H.arena);
    H = InstHost();
    set_err(b, err);
    return IRK_ERR_INVALID;
  }
  irk_status st = IRK_OK;
  cudaError_t e = cudaMemcpyAsync(H.d.u, u0, sizeof(double) * H.L,
                                  u0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(H.d.K, 0, sizeof(double) * H.s * H.L, b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dnw + k, 0, sizeof(Newton), b->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    st = IRK_ERR_CUDA;
  }
  H.used = true;
  if (st == IRK_OK) st = write_slot(b, k);
  if (st == IRK_OK && cudaStreamSynchronize(b->st) != cudaSuccess) {
    cudaGetLastError();
    st = IRK_ERR_CUDA;
  }
  if (st != IRK_OK) {
    if (H.own_arena) cudaFree(H.arena);
    H = InstHost();
    if (b->err.empty()) set_err(b, "CUDA error while admitting the instance");
    return st;
  }
  b->dirty = true;
  *slot = k;
  return IRK_OK;
}

irk_status irk_batch_step(irk_batch* b, irk_stats* stats, irk_status* status) {
  if (!b) return IRK_ERR_INVALID;
  DeviceScope ds(b->device);
  TraceRange tr("batch_step");
  int nres = 0;
  for (auto& H : b->inst) nres += H.used ? 1 : 0;
  if (stats) memset(stats, 0, sizeof(irk_stats) * b->capacity);
  if (status)
    for (int k = 0; k < b->capacity; ++k) status[k] = IRK_OK;
  if (nres == 0) return IRK_OK;
  if (b->dirty) {
    build_program(b);
    bool re = false;
    irk_status st = upload(b, &re);
    if (st != IRK_OK) return st;
    if (re || !b->exec || !(b->prog == b->captured)) {
      st = capture(b);
      if (st != IRK_OK) return st;
    }
    b->dirty = false;
  }
  BCK(cudaGraphLaunch(b->exec, b->st));
  BCK(cudaMemcpyAsync(b->hnw, b->dnw, sizeof(Newton) * b->capacity, cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  for (int k = 0; k < b->capacity; ++k) {
    if (!b->inst[k].used) continue;
    const Newton& N = b->hnw[k];
    if (stats) {
      irk_stats& s = stats[k];
      s.steps = N.status == 0 ? 1 : 0;
      s.newton_its = N.its;
      s.max_newton_its = N.its;
      s.krylov_its = N.kits;
      s.vcycles = N.vcyc;
      s.prec_apps = N.vcyc;
      s.final_rel_res = N.rel;
    }
    if (status) status[k] = (irk_status)N.status;
  }
  return IRK_OK;
}

irk_status irk_batch_get_state(irk_batch* b, int slot, double* dst, int dst_on_device) {
  if (!b || slot < 0 || slot >= b->capacity || !b->inst[slot].used || !dst) return IRK_ERR_INVALID;
  DeviceScope ds(b->device);
  const InstHost& H = b->inst[slot];
  BCK(cudaMemcpyAsync(dst, H.d.u, sizeof(double) * H.L,
                      dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  return IRK_OK;
}

irk_status irk_batch_get_stages(irk_batch* b, int slot, double* dst, int dst_on_device) {
  if (!b || slot < 0 || slot >= b->capacity || !b->inst[slot].used || !dst) return IRK_ERR_INVALID;
  DeviceScope ds(b->device);
  const InstHost& H = b->inst[slot];
  BCK(cudaMemcpyAsync(dst, H.d.K, sizeof(double) * H.s * H.L,
                      dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  return IRK_OK;
}

irk_status irk_batch_remove(irk_batch* b, int slot) {
  if (!b || slot < 0 || slot >= b->capacity || !b->inst[slot].used) return IRK_ERR_INVALID;
  DeviceScope ds(b->device);
  InstHost& H = b->inst[slot];
  cudaStreamSynchronize(b->st);
  if (H.own_arena) cudaFree(H.arena);
  H = InstHost();
  b->dirty = true;
  return IRK_OK;
}

int irk_batch_count(const irk_batch* b) {
  if (!b) return 0;
  int n = 0;
  for (auto& H : b->inst) n += H.used ? 1 : 0;
  return n;
}

const char* irk_batch_last_error(const irk_batch* b) { return b ? b->err.c_str() : ""; }

void irk_batch_destroy(irk_batch* b) {
  if (!b) return;
  DeviceScope ds(b->device);
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto& H : b->inst)
    if (H.used && H.own_arena) cudaFree(H.arena);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->dinst);
  cudaFree(b->dnw);
  cudaFree(b->dsys);
  cudaFree(b->dguard);
  cudaFree(b->dplans);
  cudaFree(b->dtasks);
  cudaFree(b->dcs);
  cudaFree(b->dctask);
  cudaFree(b->dpart);
  if (b->hnw) cudaFreeHost(b->hnw);
  if (b->aux) cudaStreamDestroy(b->aux);
  if (b->aux2) cudaStreamDestroy(b->aux2);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  cudaGetLastError();
  delete b;
}

}  // extern "C"
