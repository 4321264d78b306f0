// Matrix-free FP64 stencil kernels of the stage solve.
//
//  k_stage_states   Y_i = u_n + dt sum_j a_ij k_j (Eq. stages) and the combined
//                   fields Ybar_q = sum_m (d_q)_m Y_m that carry the s x s
//                   transform of Eq. Q0approx into every later stencil.
//  k_residual       F_i = M k_i - N(Y_i, t_n + c_i dt) (Eq. stages, Eq. dae_stage),
//                   the Algorithm-1 right-hand side -(Q0^T (x) I) F and the
//                   per-block partial sums of ||F||^2.
//  k_stage_op       Generic row operator of the transformed Jacobian:
//                   y_r = alpha base_r + sigma sum_t [m_t M x_t - dt (Jadv(Ybar_t) x_t
//                   + lin_t Jlin x_t)], used for the diagonal blocks D_i
//                   (Eq. diag_blocks), the upper coupling U (Eq. D+U) and the
//                   coupling row of L_P (Eq. Lprec).  Every N here is bilinear
//                   in the state, so sum_m d_m N'(Y_m) = Jadv(sum_m d_m Y_m) +
//                   (sum_m d_m) Jlin: the transform costs one combined field.
//  k_stage_update   k += (Q0 R0 (x) I) dk_hat (Algorithm 1 back-transform).
//  k_u_update       u_{n+1} = u_n + dt sum_i b_i k_i (Eq. update).
//
// Discretisations (periodic, h = length/n, 2D fields [y][x]):
//  Burgers-1D  N = -(u_E^2 - u_W^2)/(4h) + nu (u_E - 2u + u_W)/h^2
//  Burgers-2D  N = (-u Dx u - v Dy u + nu L u, -u Dx v - v Dy v + nu L v)
//  VSF         N = (J_A(psi, w) + nu L w, -L psi - w), M = diag(I, 0);
//              J_A is Arakawa's average of the three central Jacobians.
#include <cuda_bf16.h>

#include "irk_internal.h"

namespace irk {

__device__ __forceinline__ int wrapn(int i, int n) { return i & (n - 1); }

// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(256) k_stage_states(StageStateArgs a) {
  pdl_entry();
  const long long L = a.L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double k[S], y[S];
#pragma unroll
    for (int j = 0; j < S; ++j) k[j] = a.K[j * L + p];
    const double u = a.u ? a.u[p] : 0.0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) acc = fma(a.A[i * S + j], k[j], acc);
      y[i] = fma(a.dt, acc, u);
    }
    if (a.Y) {
#pragma unroll
      for (int i = 0; i < S; ++i) a.Y[i * L + p] = y[i];
    }
    if (a.combos) {
      for (int q = 0; q < a.ncombo; ++q) {
        double acc = 0.0;
#pragma unroll
        for (int m = 0; m < S; ++m) acc = fma(a.D[q * S + m], y[m], acc);
        a.combos[q * L + p] = acc;
      }
    }
  }
}

void launch_stage_states(const GridDesc& g, const StageStateArgs& a, cudaStream_t st) {
  const long long L = a.L;
  int blocks = (int)((L + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  switch (a.s) {
    case 1: launch_pdl(k_stage_states<1>, blocks, 256, 0, st, a); break;
    case 2: launch_pdl(k_stage_states<2>, blocks, 256, 0, st, a); break;
    case 3: launch_pdl(k_stage_states<3>, blocks, 256, 0, st, a); break;
    case 4: launch_pdl(k_stage_states<4>, blocks, 256, 0, st, a); break;
    case 5: launch_pdl(k_stage_states<5>, blocks, 256, 0, st, a); break;
  }
}

// ---------------------------------------------------------------------------
// Neighbourhood access.
struct Nbr {
  int c, e, w, n, s;              // centre, x+1, x-1, y+1, y-1
  int ne, nw, se, sw;             // diagonals (2D)
};

__device__ __forceinline__ Nbr neighbours(const GridDesc& g, int p) {
  Nbr r;
  r.c = p;
  IRK_CHECK(p, g.npts);
  if (g.dim == 1) {
    r.e = IRK_IDX(wrapn(p + 1, g.n), g.npts);
    r.w = IRK_IDX(wrapn(p - 1, g.n), g.npts);
    r.n = r.s = r.ne = r.nw = r.se = r.sw = p;
  } else {
    const int i = p & (g.n - 1), j = p >> g.logn;
    const int ip = IRK_IDX(wrapn(i + 1, g.n), g.n), im = IRK_IDX(wrapn(i - 1, g.n), g.n);
    const int jp = IRK_IDX(wrapn(j + 1, g.n), g.n), jm = IRK_IDX(wrapn(j - 1, g.n), g.n);
    IRK_CHECK(j, g.n);
    r.e = (j << g.logn) + ip;
    r.w = (j << g.logn) + im;
    r.n = (jp << g.logn) + i;
    r.s = (jm << g.logn) + i;
    r.ne = (jp << g.logn) + ip;
    r.nw = (jp << g.logn) + im;
    r.se = (jm << g.logn) + ip;
    r.sw = (jm << g.logn) + im;
  }
  return r;
}

// 3x3 neighbourhood f[dy+1][dx+1]
__device__ __forceinline__ void load9(const double* __restrict__ f, const Nbr& nb, double v[3][3]) {
  v[0][0] = __ldg(f + nb.sw); v[0][1] = __ldg(f + nb.s); v[0][2] = __ldg(f + nb.se);
  v[1][0] = __ldg(f + nb.w);  v[1][1] = __ldg(f + nb.c); v[1][2] = __ldg(f + nb.e);
  v[2][0] = __ldg(f + nb.nw); v[2][1] = __ldg(f + nb.n); v[2][2] = __ldg(f + nb.ne);
}

// Arakawa Jacobian J_A(a, b) * 12 h^2 from 3x3 neighbourhoods.
__device__ __forceinline__ double arakawa12(const double a[3][3], const double b[3][3]) {
  const double jpp = (a[1][2] - a[1][0]) * (b[2][1] - b[0][1]) - (a[2][1] - a[0][1]) * (b[1][2] - b[1][0]);
  const double jpx = a[1][2] * (b[2][2] - b[0][2]) - a[1][0] * (b[2][0] - b[0][0])
                   - a[2][1] * (b[2][2] - b[2][0]) + a[0][1] * (b[0][2] - b[0][0]);
  const double jxp = b[2][1] * (a[2][2] - a[2][0]) - b[0][1] * (a[0][2] - a[0][0])
                   - b[1][2] * (a[2][2] - a[0][2]) + b[1][0] * (a[2][0] - a[0][0]);
  return jpp + jpx + jxp;
}

__device__ __forceinline__ double lap5(const double* __restrict__ f, const Nbr& nb, int dim,
                                       double invh2) {
  if (dim == 1) return (__ldg(f + nb.e) - 2.0 * __ldg(f + nb.c) + __ldg(f + nb.w)) * invh2;
  return (__ldg(f + nb.e) + __ldg(f + nb.w) + __ldg(f + nb.n) + __ldg(f + nb.s) -
          4.0 * __ldg(f + nb.c)) * invh2;
}

// Manufactured source of the 1D operators (forcing 1):
// u*(x,t) = sin(2 pi x)(1 + 0.5 sin t) + 0.25 cos(4 pi x) cos 2t,  f = u*_t - N_h(u*).
__device__ double manufactured_source(const GridDesc& g, int p, double t) {
  const double twopi = 6.283185307179586476925286766559;
  auto ustar = [&](int q) {
    const double x = q * g.h;
    return sin(twopi * x) * (1.0 + 0.5 * sin(t)) + 0.25 * cos(2.0 * twopi * x) * cos(2.0 * t);
  };
  const double x = p * g.h;
  const double ut = 0.5 * sin(twopi * x) * cos(t) - 0.5 * cos(2.0 * twopi * x) * sin(2.0 * t);
  const double uc = ustar(p), ue = ustar(p + 1), uw = ustar(p - 1);
  double nh = g.nu * (ue - 2.0 * uc + uw) * g.invh2;
  if (g.op == IRK_OP_BURGERS_1D) nh -= (ue * ue - uw * uw) * g.inv4h;
  return ut - nh;
}

// N(Y) at point p for all components (ncomp <= 2).
template <int OP>
__device__ __forceinline__ void eval_N(const GridDesc& g, const double* __restrict__ Y, const Nbr& nb,
                                       double out[2]) {
  if (OP == IRK_OP_DIFFUSION_1D) {
    out[0] = g.nu * lap5(Y, nb, 1, g.invh2);
  } else if (OP == IRK_OP_BURGERS_1D) {
    const double ue = __ldg(Y + nb.e), uw = __ldg(Y + nb.w), uc = __ldg(Y + nb.c);
    out[0] = -(ue * ue - uw * uw) * g.inv4h + g.nu * (ue - 2.0 * uc + uw) * g.invh2;
  } else if (OP == IRK_OP_BURGERS_2D) {
    const double* u = Y;
    const double* v = Y + g.npts;
    const double uc = __ldg(u + nb.c), vc = __ldg(v + nb.c);
    const double ue = __ldg(u + nb.e), uw = __ldg(u + nb.w), un = __ldg(u + nb.n), us = __ldg(u + nb.s);
    const double ve = __ldg(v + nb.e), vw = __ldg(v + nb.w), vn = __ldg(v + nb.n), vs = __ldg(v + nb.s);
    const double ux = (ue - uw) * g.inv2h, uy = (un - us) * g.inv2h;
    const double vx = (ve - vw) * g.inv2h, vy = (vn - vs) * g.inv2h;
    const double lu = (ue + uw + un + us - 4.0 * uc) * g.invh2;
    const double lv = (ve + vw + vn + vs - 4.0 * vc) * g.invh2;
    out[0] = -uc * ux - vc * uy + g.nu * lu;
    out[1] = -uc * vx - vc * vy + g.nu * lv;
  } else {  // VSF
    double w9[3][3], p9[3][3];
    load9(Y, nb, w9);
    load9(Y + g.npts, nb, p9);
    const double lw = (w9[1][2] + w9[1][0] + w9[2][1] + w9[0][1] - 4.0 * w9[1][1]) * g.invh2;
    const double lp = (p9[1][2] + p9[1][0] + p9[2][1] + p9[0][1] - 4.0 * p9[1][1]) * g.invh2;
    out[0] = arakawa12(p9, w9) * g.inv12h2 + g.nu * lw;
    out[1] = -lp - w9[1][1];
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) r += sh[k];
  }
  return r;
}

template <int OP, int S>
__global__ void __launch_bounds__(256) k_residual(GridDesc g, ResidualArgs a) {
  pdl_entry();
  __shared__ double sh[32];
  constexpr int C = (OP == IRK_OP_BURGERS_2D || OP == IRK_OP_VSF_2D) ? 2 : 1;
  const long long L = (long long)C * g.npts;
  double sq = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.npts; p += gridDim.x * blockDim.x) {
    const Nbr nb = neighbours(g, p);
    double F[S][C];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double nv[2];
      eval_N<OP>(g, a.Y + i * L, nb, nv);
      if (a.forcing) nv[0] += manufactured_source(g, p, a.tstage[i]);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const double mass = (OP == IRK_OP_VSF_2D && c == 1) ? 0.0 : 1.0;
        const double k = a.K[i * L + c * (long long)g.npts + p];
        F[i][c] = mass * k - nv[c];
        sq = fma(F[i][c], F[i][c], sq);
      }
    }
    if (a.Fraw) {
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int c = 0; c < C; ++c) a.Fraw[i * L + c * (long long)g.npts + p] = F[i][c];
    }
    if (a.rhs) {
#pragma unroll
      for (int k = 0; k < S; ++k)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          double acc = 0.0;
#pragma unroll
          for (int i = 0; i < S; ++i) acc = fma(a.Q[i * S + k], F[i][c], acc);
          a.rhs[k * L + c * (long long)g.npts + p] = -acc;
        }
    }
  }
  const double tot = block_sum(sq, sh);
  if (threadIdx.x == 0 && a.partials) a.partials[blockIdx.x] = tot;
}

// Burgers-2D residual with one thread per point and component: half the
// per-thread state of k_residual (F for S stages of one component), twice the
// threads, and the constants folded so that N costs 10 operations per
// component:  N_c = nu/h^2 (sum of 4 neighbours - 4 f) - (u Dx + v Dy) f.
// Work item q in [0, 2 npts): component q / npts, point q % npts.
template <int S>
__global__ void __launch_bounds__(256) k_residual_b2d(GridDesc g, ResidualArgs a) {
  pdl_entry();
  __shared__ double sh[32];
  const int npts = g.npts;
  const long long L = 2LL * npts;
  const double nuh = g.nu * g.invh2, mi2h = -g.inv2h;
  double sq = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * npts; q += gridDim.x * blockDim.x) {
    const int c = (q >= npts) ? 1 : 0;
    const int p = q - c * npts;
    const Nbr nb = neighbours(g, p);
    double F[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      const double* Yi = a.Y + i * L;
      const double* f = Yi + (long long)c * npts;
      const double uc = __ldg(Yi + nb.c), vc = __ldg(Yi + npts + nb.c);
      const double fc = c ? vc : uc;
      const double fe = __ldg(f + nb.e), fw = __ldg(f + nb.w), fn = __ldg(f + nb.n), fs = __ldg(f + nb.s);
      double adv = uc * (fe - fw);
      adv = fma(vc, fn - fs, adv);
      double lap = (fe + fw) + (fn + fs);
      lap = fma(-4.0, fc, lap);
      const double nv = fma(nuh, lap, mi2h * adv);
      F[i] = __ldg(a.K + i * L + q) - nv;
      sq = fma(F[i], F[i], sq);
    }
    if (a.Fraw) {
#pragma unroll
      for (int i = 0; i < S; ++i) a.Fraw[i * L + q] = F[i];
    }
    if (a.rhs) {
#pragma unroll
      for (int k = 0; k < S; ++k) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < S; ++i) acc = fma(-a.Q[i * S + k], F[i], acc);
        a.rhs[k * L + q] = acc;
      }
    }
  }
  const double tot = block_sum(sq, sh);
  if (threadIdx.x == 0 && a.partials) a.partials[blockIdx.x] = tot;
}

// VSF residual with one thread per point and component (as k_residual_b2d):
// the vorticity item forms J_A(psi, w) + nu L w (M = 1), the streamfunction
// item the constraint row -L psi - w (M = 0).
template <int S>
__global__ void __launch_bounds__(256) k_residual_vsf(GridDesc g, ResidualArgs a) {
  pdl_entry();
  __shared__ double sh[32];
  const int npts = g.npts;
  const long long L = 2LL * npts;
  double sq = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * npts; q += gridDim.x * blockDim.x) {
    const int c = (q >= npts) ? 1 : 0;
    const int p = q - c * npts;
    const Nbr nb = neighbours(g, p);
    double F[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      const double* Yw = a.Y + i * L;
      const double* Yp = Yw + npts;
      double nv;
      if (c == 0) {
        double w9[3][3], p9[3][3];
        load9(Yw, nb, w9);
        load9(Yp, nb, p9);
        const double lw = (w9[1][2] + w9[1][0] + w9[2][1] + w9[0][1] - 4.0 * w9[1][1]) * g.invh2;
        nv = arakawa12(p9, w9) * g.inv12h2 + g.nu * lw;
        F[i] = __ldg(a.K + i * L + q) - nv;
      } else {
        const double lp = (__ldg(Yp + nb.e) + __ldg(Yp + nb.w) + __ldg(Yp + nb.n) +
                           __ldg(Yp + nb.s) - 4.0 * __ldg(Yp + nb.c)) * g.invh2;
        nv = -lp - __ldg(Yw + nb.c);
        F[i] = -nv;
      }
      sq = fma(F[i], F[i], sq);
    }
    if (a.Fraw) {
#pragma unroll
      for (int i = 0; i < S; ++i) a.Fraw[i * L + q] = F[i];
    }
    if (a.rhs) {
#pragma unroll
      for (int k = 0; k < S; ++k) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < S; ++i) acc = fma(-a.Q[i * S + k], F[i], acc);
        a.rhs[k * L + q] = acc;
      }
    }
  }
  const double tot = block_sum(sq, sh);
  if (threadIdx.x == 0 && a.partials) a.partials[blockIdx.x] = tot;
}

int residual_blocks(const GridDesc& g) {
  const long long items = (g.op == IRK_OP_BURGERS_2D || g.op == IRK_OP_VSF_2D) ? 2LL * g.npts : g.npts;
  int blocks = (int)((items + 255) / 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  return blocks;
}

template <int OP>
static void launch_residual_op(const GridDesc& g, const ResidualArgs& a, cudaStream_t st) {
  const int blocks = residual_blocks(g);
  if (OP == IRK_OP_BURGERS_2D && !a.forcing) {
    switch (a.s) {
      case 1: launch_pdl(k_residual_b2d<1>, blocks, 256, 0, st, g, a); break;
      case 2: launch_pdl(k_residual_b2d<2>, blocks, 256, 0, st, g, a); break;
      case 3: launch_pdl(k_residual_b2d<3>, blocks, 256, 0, st, g, a); break;
      case 4: launch_pdl(k_residual_b2d<4>, blocks, 256, 0, st, g, a); break;
      case 5: launch_pdl(k_residual_b2d<5>, blocks, 256, 0, st, g, a); break;
    }
    return;
  }
  if (OP == IRK_OP_VSF_2D && !a.forcing) {
    switch (a.s) {
      case 1: launch_pdl(k_residual_vsf<1>, blocks, 256, 0, st, g, a); break;
      case 2: launch_pdl(k_residual_vsf<2>, blocks, 256, 0, st, g, a); break;
      case 3: launch_pdl(k_residual_vsf<3>, blocks, 256, 0, st, g, a); break;
      case 4: launch_pdl(k_residual_vsf<4>, blocks, 256, 0, st, g, a); break;
      case 5: launch_pdl(k_residual_vsf<5>, blocks, 256, 0, st, g, a); break;
    }
    return;
  }
  switch (a.s) {
    case 1: launch_pdl(k_residual<OP, 1>, blocks, 256, 0, st, g, a); break;
    case 2: launch_pdl(k_residual<OP, 2>, blocks, 256, 0, st, g, a); break;
    case 3: launch_pdl(k_residual<OP, 3>, blocks, 256, 0, st, g, a); break;
    case 4: launch_pdl(k_residual<OP, 4>, blocks, 256, 0, st, g, a); break;
    case 5: launch_pdl(k_residual<OP, 5>, blocks, 256, 0, st, g, a); break;
  }
}

void launch_residual(const GridDesc& g, const ResidualArgs& a, cudaStream_t st) {
  switch (g.op) {
    case IRK_OP_DIFFUSION_1D: launch_residual_op<IRK_OP_DIFFUSION_1D>(g, a, st); break;
    case IRK_OP_BURGERS_1D: launch_residual_op<IRK_OP_BURGERS_1D>(g, a, st); break;
    case IRK_OP_BURGERS_2D: launch_residual_op<IRK_OP_BURGERS_2D>(g, a, st); break;
    case IRK_OP_VSF_2D: launch_residual_op<IRK_OP_VSF_2D>(g, a, st); break;
  }
}

// ---------------------------------------------------------------------------
// One term of the row operator at point p, accumulated into acc[c]:
//   m M x - dt (Jadv(Ybar) x + lin Jlin x)
// WONLY (VSF only): x, y and base hold the vorticity alone (the stream
// function parts are absent): the J_A(x_psi, wbar) coupling and the psi row
// are dropped, which is the omega block of the Picard system Eq. vsf-system-2.
template <int OP, bool WONLY = false>
__device__ __forceinline__ void term_apply(const GridDesc& g, const OpTerm& t, const Nbr& nb,
                                           double dt, double acc[2]) {
  const int npts = g.npts;
  if (!t.combo && t.lin == 0.0) {  // mass term only: no neighbours needed
    acc[0] = fma(t.m, __ldg(t.x + nb.c), acc[0]);
    if (OP == IRK_OP_BURGERS_2D) acc[1] = fma(t.m, __ldg(t.x + npts + nb.c), acc[1]);
    return;
  }
  if (OP == IRK_OP_DIFFUSION_1D || OP == IRK_OP_BURGERS_1D) {
    const double* x = t.x;
    const double xc = __ldg(x + nb.c), xe = __ldg(x + nb.e), xw = __ldg(x + nb.w);
    double op = 0.0;
    if (OP == IRK_OP_BURGERS_1D && t.combo)
      op = -(__ldg(t.combo + nb.e) * xe - __ldg(t.combo + nb.w) * xw) * g.inv2h;
    if (t.lin != 0.0) op = fma(t.lin * g.nu, (xe - 2.0 * xc + xw) * g.invh2, op);
    acc[0] += t.m * xc - dt * op;
  } else if (OP == IRK_OP_BURGERS_2D && t.coef) {
    // coefficient form with the combined field's coefficients precomputed
    // (k_combo_coef): 20 FP64 operations per point instead of 30
    const double* f = t.coef + nb.c;
    const double AX = __ldg(f), AY = __ldg(f + npts), DU = __ldg(f + 2 * npts);
    const double XUV = __ldg(f + 3 * npts), XVU = __ldg(f + 4 * npts), DV = __ldg(f + 5 * npts);
    const double kd = t.kd, cc = t.cc;  // uniform, formed on the host
    const double ce = AX - kd, cw = -AX - kd, cn = AY - kd, cs = -AY - kd;
    const double* xu = t.x;
    const double* xv = t.x + npts;
    const double uc = __ldg(xu + nb.c), vc = __ldg(xv + nb.c);
    double yu = fma(cc + DU, uc, XUV * vc);
    yu = fma(ce, __ldg(xu + nb.e), yu);
    yu = fma(cw, __ldg(xu + nb.w), yu);
    yu = fma(cn, __ldg(xu + nb.n), yu);
    yu = fma(cs, __ldg(xu + nb.s), yu);
    double yv = fma(cc + DV, vc, XVU * uc);
    yv = fma(ce, __ldg(xv + nb.e), yv);
    yv = fma(cw, __ldg(xv + nb.w), yv);
    yv = fma(cn, __ldg(xv + nb.n), yv);
    yv = fma(cs, __ldg(xv + nb.s), yv);
    acc[0] += yu;
    acc[1] += yv;
  } else if (OP == IRK_OP_BURGERS_2D && t.combo && t.lin != 0.0) {
    // Diagonal term in coefficient form.  For component u:
    //   m x_u - dt (-(x_u ub_x + ub Dx x_u + x_v ub_y + vb Dy x_u) + lin nu L x_u)
    //   = (m + dt ub_x + 4 k) x_u + dt ub_y x_v + sum_K c_K x_u(K),
    // with k = dt lin nu / h^2, c_E/W = +-dt ub/(2h) - k, c_N/S = +-dt vb/(2h) - k;
    // the neighbour coefficients are shared by both components.
    const double* bu = t.combo;
    const double* bv = t.combo + npts;
    const double ax = dt * g.inv2h * __ldg(bu + nb.c), ay = dt * g.inv2h * __ldg(bv + nb.c);
    const double kd = dt * t.lin * g.nu * g.invh2;
    const double ce = ax - kd, cw = -ax - kd, cn = ay - kd, cs = -ay - kd;
    const double dth = dt * g.inv2h;
    const double bux = dth * (__ldg(bu + nb.e) - __ldg(bu + nb.w));
    const double buy = dth * (__ldg(bu + nb.n) - __ldg(bu + nb.s));
    const double bvx = dth * (__ldg(bv + nb.e) - __ldg(bv + nb.w));
    const double bvy = dth * (__ldg(bv + nb.n) - __ldg(bv + nb.s));
    const double cc = t.m + 4.0 * kd;
    const double* xu = t.x;
    const double* xv = t.x + npts;
    const double uc = __ldg(xu + nb.c), vc = __ldg(xv + nb.c);
    double yu = fma(cc + bux, uc, buy * vc);
    yu = fma(ce, __ldg(xu + nb.e), yu);
    yu = fma(cw, __ldg(xu + nb.w), yu);
    yu = fma(cn, __ldg(xu + nb.n), yu);
    yu = fma(cs, __ldg(xu + nb.s), yu);
    double yv = fma(cc + bvy, vc, bvx * uc);
    yv = fma(ce, __ldg(xv + nb.e), yv);
    yv = fma(cw, __ldg(xv + nb.w), yv);
    yv = fma(cn, __ldg(xv + nb.n), yv);
    yv = fma(cs, __ldg(xv + nb.s), yv);
    acc[0] += yu;
    acc[1] += yv;
  } else if (OP == IRK_OP_BURGERS_2D) {
    const double* xu = t.x;
    const double* xv = t.x + npts;
    const double uc = __ldg(xu + nb.c), ue = __ldg(xu + nb.e), uw = __ldg(xu + nb.w),
                 un = __ldg(xu + nb.n), us = __ldg(xu + nb.s);
    const double vc = __ldg(xv + nb.c), ve = __ldg(xv + nb.e), vw = __ldg(xv + nb.w),
                 vn = __ldg(xv + nb.n), vs = __ldg(xv + nb.s);
    double opu = 0.0, opv = 0.0;
    if (t.combo) {
      const double* bu = t.combo;
      const double* bv = t.combo + npts;
      const double buc = __ldg(bu + nb.c), bvc = __ldg(bv + nb.c);
      const double bux = (__ldg(bu + nb.e) - __ldg(bu + nb.w)) * g.inv2h;
      const double buy = (__ldg(bu + nb.n) - __ldg(bu + nb.s)) * g.inv2h;
      const double bvx = (__ldg(bv + nb.e) - __ldg(bv + nb.w)) * g.inv2h;
      const double bvy = (__ldg(bv + nb.n) - __ldg(bv + nb.s)) * g.inv2h;
      const double xux = (ue - uw) * g.inv2h, xuy = (un - us) * g.inv2h;
      const double xvx = (ve - vw) * g.inv2h, xvy = (vn - vs) * g.inv2h;
      opu = -(uc * bux + buc * xux + vc * buy + bvc * xuy);
      opv = -(uc * bvx + buc * xvx + vc * bvy + bvc * xvy);
    }
    if (t.lin != 0.0) {
      const double k = t.lin * g.nu * g.invh2;
      opu = fma(k, ue + uw + un + us - 4.0 * uc, opu);
      opv = fma(k, ve + vw + vn + vs - 4.0 * vc, opv);
    }
    acc[0] += t.m * uc - dt * opu;
    acc[1] += t.m * vc - dt * opv;
  } else if (t.coef) {  // VSF with the combined field's Arakawa weights precomputed
    double xw9[3][3], xp9[3][3];
    load9(t.x, nb, xw9);
    if (!WONLY) load9(t.x + npts, nb, xp9);
    const double* f = t.coef + nb.c;
    const long long st = npts;
    // -dt (J_A(psibar, xw) + J_A(xp, wbar)) in 16 FMAs, order E, W, N, S, NE, NW, SE, SW
    double op = __ldg(f) * xw9[1][2];
    op = fma(__ldg(f + st), xw9[1][0], op);
    op = fma(__ldg(f + 2 * st), xw9[2][1], op);
    op = fma(__ldg(f + 3 * st), xw9[0][1], op);
    op = fma(__ldg(f + 4 * st), xw9[2][2], op);
    op = fma(__ldg(f + 5 * st), xw9[2][0], op);
    op = fma(__ldg(f + 6 * st), xw9[0][2], op);
    op = fma(__ldg(f + 7 * st), xw9[0][0], op);
    if (!WONLY) {
      op = fma(__ldg(f + 8 * st), xp9[1][2], op);
      op = fma(__ldg(f + 9 * st), xp9[1][0], op);
      op = fma(__ldg(f + 10 * st), xp9[2][1], op);
      op = fma(__ldg(f + 11 * st), xp9[0][1], op);
      op = fma(__ldg(f + 12 * st), xp9[2][2], op);
      op = fma(__ldg(f + 13 * st), xp9[2][0], op);
      op = fma(__ldg(f + 14 * st), xp9[0][2], op);
      op = fma(__ldg(f + 15 * st), xp9[0][0], op);
    }
    double opp = 0.0;
    if (t.lin != 0.0) {
      const double lw = (xw9[1][2] + xw9[1][0] + xw9[2][1] + xw9[0][1] - 4.0 * xw9[1][1]) * g.invh2;
      op = fma(-dt * t.lin * g.nu, lw, op);
      if (!WONLY) {
        const double lp = (xp9[1][2] + xp9[1][0] + xp9[2][1] + xp9[0][1] - 4.0 * xp9[1][1]) * g.invh2;
        opp = t.lin * (-xw9[1][1] - lp);
      }
    }
    acc[0] += t.m * xw9[1][1] + op;
    if (!WONLY) acc[1] += -dt * opp;
  } else {  // VSF: state (w, psi), M = diag(1, 0)
    double xw9[3][3], xp9[3][3];
    load9(t.x, nb, xw9);
    if (!WONLY) load9(t.x + npts, nb, xp9);
    double opw = 0.0, opp = 0.0;
    if (t.combo) {
      double bw9[3][3], bp9[3][3];
      load9(t.combo + npts, nb, bp9);
      if (WONLY) {
        opw = arakawa12(bp9, xw9) * g.inv12h2;
      } else {
        load9(t.combo, nb, bw9);
        opw = (arakawa12(bp9, xw9) + arakawa12(xp9, bw9)) * g.inv12h2;
      }
    }
    if (t.lin != 0.0) {
      const double lw = (xw9[1][2] + xw9[1][0] + xw9[2][1] + xw9[0][1] - 4.0 * xw9[1][1]) * g.invh2;
      opw = fma(t.lin * g.nu, lw, opw);
      if (!WONLY) {
        const double lp = (xp9[1][2] + xp9[1][0] + xp9[2][1] + xp9[0][1] - 4.0 * xp9[1][1]) * g.invh2;
        opp = t.lin * (-xw9[1][1] - lp);
      }
    }
    acc[0] += t.m * xw9[1][1] - dt * opw;
    if (!WONLY) acc[1] += -dt * opp;
  }
}

template <int OP, bool WONLY = false>
__global__ void __launch_bounds__(256) k_stage_op(GridDesc g, StageOpArgs a) {
  pdl_entry();
  constexpr int C = WONLY ? 1 : (OP == IRK_OP_BURGERS_2D || OP == IRK_OP_VSF_2D) ? 2 : 1;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.npts; p += gridDim.x * blockDim.x) {
    const Nbr nb = neighbours(g, p);
    for (int r = 0; r < a.nrow; ++r) {
      const OpRow& row = a.row[r];
      double acc[2] = {0.0, 0.0};
      for (int k = 0; k < row.nterm; ++k) term_apply<OP, WONLY>(g, row.t[k], nb, a.dt, acc);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const long long idx = (long long)c * g.npts + p;
        double y = row.sigma * acc[c];
        if (row.base) y = fma(row.alpha, row.base[idx], y);
        row.y[idx] = y;
      }
    }
    if (a.copy_dst) {
      double* dst = a.copy_dst;
      if (a.copy_jdev) dst += (long long)(*a.copy_jdev) * a.copy_ldv;
      for (long long q = p; q < a.copy_len; q += g.npts) dst[q] = a.copy_src[q];
    }
  }
}

__global__ void __launch_bounds__(256) k_combo_coef(GridDesc g, const double* __restrict__ combos,
                                                    ComboList list, double dt, double* __restrict__ coef) {
  pdl_entry();
  const int ncombo = list.n;
  const int npts = g.npts;
  const double dth = dt * g.inv2h;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npts; p += gridDim.x * blockDim.x) {
    const Nbr nb = neighbours(g, p);
#pragma unroll 1
    for (int q = 0; q < ncombo; ++q) {
      const double* bu = combos + (long long)list.idx[q] * 2 * npts;
      const double* bv = bu + npts;
      double* f = coef + (long long)q * 6 * npts + p;
      f[0] = dth * __ldg(bu + nb.c);
      f[npts] = dth * __ldg(bv + nb.c);
      f[2 * npts] = dth * (__ldg(bu + nb.e) - __ldg(bu + nb.w));
      f[3 * npts] = dth * (__ldg(bu + nb.n) - __ldg(bu + nb.s));
      f[4 * npts] = dth * (__ldg(bv + nb.e) - __ldg(bv + nb.w));
      f[5 * npts] = dth * (__ldg(bv + nb.n) - __ldg(bv + nb.s));
    }
  }
}

// The Arakawa Jacobian J_A(a, b) is linear in b with an 8-point stencil whose
// weights depend on a (no centre weight), and antisymmetric: J_A(x, b) =
// -J_A(b, x).  Weights of b (times 12 h^2), in the order E, W, N, S, NE, NW,
// SE, SW, from the three central forms of Arakawa's average.
__device__ __forceinline__ void arakawa_weights(const double a[3][3], double wgt[8]) {
  const double aE = a[1][2], aW = a[1][0], aN = a[2][1], aS = a[0][1];
  const double aNE = a[2][2], aNW = a[2][0], aSE = a[0][2], aSW = a[0][0];
  wgt[0] = -(aN - aS) - (aNE - aSE);  // E
  wgt[1] = (aN - aS) + (aNW - aSW);   // W
  wgt[2] = (aE - aW) + (aNE - aNW);   // N
  wgt[3] = -(aE - aW) - (aSE - aSW);  // S
  wgt[4] = aE - aN;                   // NE
  wgt[5] = aN - aW;                   // NW
  wgt[6] = aS - aE;                   // SE
  wgt[7] = aW - aS;                   // SW
}

// VSF: 16 fields per combined field (wbar, psibar): P_k = -dt/(12h^2) times the
// weights of J_A(psibar, .) (applied to x_omega) and Q_k = +dt/(12h^2) times
// the weights of J_A(wbar, .) (applied to x_psi, by antisymmetry), so that
// sum_k P_k xw_k + Q_k xp_k = -dt (J_A(psibar, xw) + J_A(xp, wbar)).
// One work item per (combined field, half, point): half 0 forms P from psibar,
// half 1 forms Q from wbar (write-bound: 64 bytes per item).
__global__ void __launch_bounds__(256) k_combo_coef_vsf(GridDesc g, const double* __restrict__ combos,
                                                        ComboList list, double dt, double* __restrict__ coef) {
  pdl_entry();
  const int npts = g.npts, ncombo = list.n;
  const double sc = dt * g.inv12h2;
  const long long items = 2LL * ncombo * npts;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(it % npts);
    const long long qh = it / npts;  // 2 q + half
    const int q = (int)(qh >> 1), half = (int)(qh & 1);
    const Nbr nb = neighbours(g, p);
    const double* src = combos + (long long)list.idx[q] * 2 * npts + (half ? 0 : npts);  // psibar | wbar
    double a9[3][3], wgt[8];
    load9(src, nb, a9);
    arakawa_weights(a9, wgt);
    const double scl = half ? sc : -sc;
    double* f = coef + (long long)q * 16 * npts + (long long)half * 8 * npts + p;
#pragma unroll
    for (int k = 0; k < 8; ++k) f[(long long)k * npts] = scl * wgt[k];
  }
}

int combo_coef_fields(int op) {
  return op == IRK_OP_BURGERS_2D ? 6 : (op == IRK_OP_VSF_2D ? 16 : 0);
}

void launch_combo_coef(const GridDesc& g, const double* combos, const ComboList& list, double dt,
                       double* coef, cudaStream_t st) {
  if (list.n <= 0) return;
  int blocks = (g.npts + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (g.op == IRK_OP_VSF_2D)
    launch_pdl(k_combo_coef_vsf, 152 * 8, 256, 0, st, g, combos, list, dt, coef);
  else
    launch_pdl(k_combo_coef, blocks, 256, 0, st, g, combos, list, dt, coef);
}

void launch_stage_op(const GridDesc& g, const StageOpArgs& a_in, cudaStream_t st) {
  StageOpArgs a = a_in;
  for (int r = 0; r < a.nrow; ++r)
    for (int t = 0; t < a.row[r].nterm; ++t) {
      OpTerm& tm = a.row[r].t[t];
      tm.kd = a.dt * tm.lin * g.nu * g.invh2;
      tm.cc = tm.m + 4.0 * tm.kd;
    }
  int blocks = (g.npts + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  switch (g.op) {
    case IRK_OP_DIFFUSION_1D: launch_pdl(k_stage_op<IRK_OP_DIFFUSION_1D>, blocks, 256, 0, st, g, a); break;
    case IRK_OP_BURGERS_1D: launch_pdl(k_stage_op<IRK_OP_BURGERS_1D>, blocks, 256, 0, st, g, a); break;
    case IRK_OP_BURGERS_2D: launch_pdl(k_stage_op<IRK_OP_BURGERS_2D>, blocks, 256, 0, st, g, a); break;
    case IRK_OP_VSF_2D:
      if (a.vsf_omega_only) launch_pdl(k_stage_op<IRK_OP_VSF_2D, true>, blocks, 256, 0, st, g, a);
      else launch_pdl(k_stage_op<IRK_OP_VSF_2D>, blocks, 256, 0, st, g, a);
      break;
  }
}

// y = -L_h x (5-point, periodic, 2D): the stream function rows of Eq.
// vsf-system-2 divided by -dt, for the Poisson FGMRES of the forward solve.
__global__ void __launch_bounds__(256) k_neg_laplacian_2d(GridDesc g, const double* __restrict__ x,
                                                          double* __restrict__ y) {
  pdl_entry();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.npts; p += gridDim.x * blockDim.x) {
    const Nbr nb = neighbours(g, p);
    y[p] = (4.0 * __ldg(x + nb.c) - __ldg(x + nb.e) - __ldg(x + nb.w) - __ldg(x + nb.n) -
            __ldg(x + nb.s)) * g.invh2;
  }
}

void launch_neg_laplacian(const GridDesc& g, const double* x, double* y, cudaStream_t st) {
  int blocks = (g.npts + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  launch_pdl(k_neg_laplacian_2d, blocks, 256, 0, st, g, x, y);
}

// ---------------------------------------------------------------------------
struct SmallMat {
  double m[IRK_MAXS * IRK_MAXS];
};

template <int S>
__global__ void __launch_bounds__(256) k_stage_update(long long L, SmallMat T, const double* __restrict__ yhat,
                                                      double* __restrict__ K) {
  pdl_entry();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double y[S];
#pragma unroll
    for (int k = 0; k < S; ++k) y[k] = yhat[k * L + p];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double acc = K[i * L + p];
#pragma unroll
      for (int k = 0; k < S; ++k) acc = fma(T.m[i * S + k], y[k], acc);
      K[i * L + p] = acc;
    }
  }
}

// Newton starting value from the previous step's stages (in place; E read
// from device memory, so one captured graph follows the host's choice of E)
template <int S>
__global__ void __launch_bounds__(256) k_stage_extrapolate(long long L, const double* __restrict__ E,
                                                           double* __restrict__ K) {
  pdl_entry();
  __shared__ double e[S * S];
  for (int i = threadIdx.x; i < S * S; i += blockDim.x) e[i] = E[i];
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double k[S];
#pragma unroll
    for (int i = 0; i < S; ++i) k[i] = K[i * L + p];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < S; ++i) acc = fma(e[j * S + i], k[i], acc);
      K[j * L + p] = acc;
    }
  }
}

void launch_stage_extrapolate(long long L, int s, const double* E, double* K, cudaStream_t st) {
  int blocks = (int)((L + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  switch (s) {
    case 1: launch_pdl(k_stage_extrapolate<1>, blocks, 256, 0, st, L, E, K); break;
    case 2: launch_pdl(k_stage_extrapolate<2>, blocks, 256, 0, st, L, E, K); break;
    case 3: launch_pdl(k_stage_extrapolate<3>, blocks, 256, 0, st, L, E, K); break;
    case 4: launch_pdl(k_stage_extrapolate<4>, blocks, 256, 0, st, L, E, K); break;
    case 5: launch_pdl(k_stage_extrapolate<5>, blocks, 256, 0, st, L, E, K); break;
  }
}

void launch_stage_update(long long L, int s, const double* QR, const double* yhat, double* K,
                         cudaStream_t st) {
  SmallMat T;
  for (int i = 0; i < s * s; ++i) T.m[i] = QR[i];
  int blocks = (int)((L + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  switch (s) {
    case 1: launch_pdl(k_stage_update<1>, blocks, 256, 0, st, L, T, yhat, K); break;
    case 2: launch_pdl(k_stage_update<2>, blocks, 256, 0, st, L, T, yhat, K); break;
    case 3: launch_pdl(k_stage_update<3>, blocks, 256, 0, st, L, T, yhat, K); break;
    case 4: launch_pdl(k_stage_update<4>, blocks, 256, 0, st, L, T, yhat, K); break;
    case 5: launch_pdl(k_stage_update<5>, blocks, 256, 0, st, L, T, yhat, K); break;
  }
}

template <int S>
__global__ void __launch_bounds__(256) k_u_update(long long L, SmallMat bw, const double* __restrict__ K,
                                                  double* __restrict__ u) {
  pdl_entry();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < S; ++i) acc = fma(bw.m[i], K[i * L + p], acc);
    u[p] = fma(bw.m[IRK_MAXS], acc, u[p]);
  }
}

void launch_u_update(long long L, int s, const double* b, double dt, const double* K, double* u,
                     cudaStream_t st) {
  SmallMat bw;
  for (int i = 0; i < s; ++i) bw.m[i] = b[i];
  bw.m[IRK_MAXS] = dt;
  int blocks = (int)((L + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  switch (s) {
    case 1: launch_pdl(k_u_update<1>, blocks, 256, 0, st, L, bw, K, u); break;
    case 2: launch_pdl(k_u_update<2>, blocks, 256, 0, st, L, bw, K, u); break;
    case 3: launch_pdl(k_u_update<3>, blocks, 256, 0, st, L, bw, K, u); break;
    case 4: launch_pdl(k_u_update<4>, blocks, 256, 0, st, L, bw, K, u); break;
    case 5: launch_pdl(k_u_update<5>, blocks, 256, 0, st, L, bw, K, u); break;
  }
}

// ---------------------------------------------------------------------------
// Multigrid coefficient field of a diagonal block row: the advecting
// velocity of the frozen-coefficient operator.  Burgers: the combined state
// itself; VSF: (Dy psibar, -Dx psibar).  Written in the MG storage precision.
template <typename T>
__device__ __forceinline__ void store_as(T* p, double v);
template <>
__device__ __forceinline__ void store_as<double>(double* p, double v) { *p = v; }
template <>
__device__ __forceinline__ void store_as<float>(float* p, double v) { *p = (float)v; }
template <>
__device__ __forceinline__ void store_as<__nv_bfloat16>(__nv_bfloat16* p, double v) {
  *p = __double2bfloat16(v);
}

template <typename T>
__global__ void k_velocity(GridDesc g, const double* __restrict__ combo, T* __restrict__ vel) {
  pdl_entry();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.npts; p += gridDim.x * blockDim.x) {
    if (g.op == IRK_OP_VSF_2D) {
      const Nbr nb = neighbours(g, p);
      const double* psi = combo + g.npts;
      store_as<T>(vel + p, (__ldg(psi + nb.n) - __ldg(psi + nb.s)) * g.inv2h);
      store_as<T>(vel + g.npts + p, -(__ldg(psi + nb.e) - __ldg(psi + nb.w)) * g.inv2h);
    } else if (g.op == IRK_OP_BURGERS_2D) {
      store_as<T>(vel + p, combo[p]);
      store_as<T>(vel + g.npts + p, combo[g.npts + p]);
    } else if (g.op == IRK_OP_BURGERS_1D) {
      store_as<T>(vel + p, combo[p]);
    } else {
      store_as<T>(vel + p, 0.0);
    }
  }
}

void launch_velocity_from_combo(const GridDesc& g, const double* combo, void* vel, int prec,
                                cudaStream_t st) {
  int blocks = (g.npts + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (prec == IRK_MG_FP64)
    launch_pdl(k_velocity<double>, blocks, 256, 0, st, g, combo, (double*)vel);
  else if (prec == IRK_MG_FP32)
    launch_pdl(k_velocity<float>, blocks, 256, 0, st, g, combo, (float*)vel);
  else
    launch_pdl(k_velocity<__nv_bfloat16>, blocks, 256, 0, st, g, combo, (__nv_bfloat16*)vel);
}

// ---------------------------------------------------------------------------
// Zero-mean projection of periodic fields (the psi null space of the DAE).
__global__ void k_field_sums(long long npts, long long stride, const double* __restrict__ x,
                             double* __restrict__ partials) {
  pdl_entry();
  __shared__ double sh[32];
  const double* f = x + blockIdx.y * stride;
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts;
       p += (long long)gridDim.x * blockDim.x)
    acc += f[p];
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

__global__ void k_field_sub_mean(long long npts, long long stride, int nblk,
                                 const double* __restrict__ partials, double* __restrict__ x) {
  pdl_entry();
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partials[blockIdx.y * nblk + b];
    mean = s / (double)npts;
  }
  __syncthreads();
  double* f = x + blockIdx.y * stride;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts;
       p += (long long)gridDim.x * blockDim.x)
    f[p] -= mean;
}

void launch_remove_mean(long long npts, int nfields, long long stride, double* x, double* scratch,
                        cudaStream_t st) {
  int nblk = (int)((npts + 255) / 256);
  if (nblk > 152) nblk = 152;
  dim3 grid(nblk, nfields);
  launch_pdl(k_field_sums, grid, 256, 0, st, npts, stride, x, scratch);
  launch_pdl(k_field_sub_mean, grid, 256, 0, st, npts, stride, nblk, scratch, x);
}

}  // namespace irk

IRK_BOUNDS_TU(stencil)
