// Geometric multigrid V-cycle kernels (steps a9/a10): one V-cycle stands in
// for each inner inverse (gamma M - dt L)^{-1} of the block preconditioner
// L_P (Eq. Lprec; inexact inner inverses as in Sec. 4).
//
// Scalar operator per state component on a periodic grid with spacing h:
//   A w = sigma w + cadv * adv(a, w) - cdiff * L_h w
//   MG_ADVECTIVE        adv = a_x Dx w + a_y Dy w   (central; 2D or 1D)
//   MG_CONSERVATIVE_1D  adv = (a_E w_E - a_W w_W) / (2h)
//   MG_DIFFUSION        adv = 0 (cadv ignored)
// The velocity a is the frozen combined field of the block row, restricted
// to every level by full weighting; coarse operators are rediscretised at 2h.
// Smoother: damped Jacobi; transfers: full weighting and (bi)linear
// interpolation on vertex-centred grids (coarse point I = fine point 2I);
// coarsest level: Jacobi sweeps in one CTA out of shared memory.
//
// Storage precision: double (FP64), float (FP32) or bf16 with float
// arithmetic (BF16-stored data, FP32 accumulation).
#include <cuda_bf16.h>

#include <cstring>

#include "irk_internal.h"
#include <cstdlib>
#include <type_traits>

namespace irk {

template <typename TS> struct Cmp { typedef float T; };
template <> struct Cmp<double> { typedef double T; };

template <typename TS>
__device__ __forceinline__ typename Cmp<TS>::T ldv(const TS* p) { return *p; }
template <>
__device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <typename TS, typename TC>
__device__ __forceinline__ void stv(TS* p, TC v) { *p = (TS)v; }
template <>
__device__ __forceinline__ void stv<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

struct LvIdx {
  int c, e, w, n, s;
};

template <int DIM>
__device__ __forceinline__ LvIdx lv_nbr(const MGLevelDesc& lv, int p) {
  LvIdx r;
  r.c = p;
  const int m = lv.n - 1;
  IRK_CHECK(p, lv.npts);
  if (DIM == 1) {
    r.e = IRK_IDX((p + 1) & m, lv.npts);
    r.w = IRK_IDX((p - 1) & m, lv.npts);
    r.n = r.s = p;
  } else {
    const int i = p & m, j = p >> lv.logn;
    r.e = IRK_IDX((j << lv.logn) + ((i + 1) & m), lv.npts);
    r.w = IRK_IDX((j << lv.logn) + ((i - 1) & m), lv.npts);
    r.n = IRK_IDX((((j + 1) & m) << lv.logn) + i, lv.npts);
    r.s = IRK_IDX((((j - 1) & m) << lv.logn) + i, lv.npts);
  }
  return r;
}

// Grid point (gx, gy) of a level with n = 2^ln points per side (2D tile kernels)
__device__ __forceinline__ int tile_pt(int gx, int gy, int ln, int n) {
  return ((int)IRK_IDX(gy, n) << ln) + (int)IRK_IDX(gx, n);
}

// Stencil of A at one point in coefficient form, A w = D w_c + sum_k c_k w_k
// over the neighbours k (E, W, N, S).  The four coefficients depend only on
// the velocity, so they are formed once per point and shared by all
// components; the Jacobi update then costs one FMA per neighbour.
template <typename TC>
struct Coef4 {
  TC e, w, n, s;
};

template <typename TS, int DIM, int KIND, typename TV = TS>
__device__ __forceinline__ Coef4<typename Cmp<TS>::T> stencil_coef(
    const LvIdx& q, const TV* __restrict__ vel, int npts, typename Cmp<TS>::T alpha,
    typename Cmp<TS>::T beta) {
  // alpha = cadv / (2h), beta = -cdiff / h^2 (off-diagonal diffusion weight)
  typedef typename Cmp<TS>::T TC;
  Coef4<TC> c;
  c.e = c.w = c.n = c.s = beta;
  if (KIND == MG_ADVECTIVE) {
    const TC ax = ldv(vel + q.c);
    c.e = fma(alpha, ax, beta);
    c.w = fma(-alpha, ax, beta);
    if (DIM == 2) {
      const TC ay = ldv(vel + npts + q.c);
      c.n = fma(alpha, ay, beta);
      c.s = fma(-alpha, ay, beta);
    }
  } else if (KIND == MG_CONSERVATIVE_1D) {
    c.e = fma(alpha, ldv(vel + q.e), beta);
    c.w = fma(-alpha, ldv(vel + q.w), beta);
  } else if (KIND == MG_ADVECTIVE_PRE) {  // 2D, coefficients precomputed
    c.e = ldv(vel + q.c);
    c.w = ldv(vel + npts + q.c);
    c.n = ldv(vel + 2 * npts + q.c);
    c.s = ldv(vel + 3 * npts + q.c);
  }
  return c;
}

template <typename TS>
__global__ void __launch_bounds__(256) k_mg_coef(MGLevelDesc lv, double alpha64, double beta64,
                                                 const TS* __restrict__ vel, TS* __restrict__ coef) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  const TC alpha = TC(alpha64), beta = TC(beta64);
  const int npts = lv.npts;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npts; p += gridDim.x * blockDim.x) {
    const TC ax = ldv(vel + p), ay = ldv(vel + npts + p);
    stv<TS, TC>(coef + p, fma(alpha, ax, beta));
    stv<TS, TC>(coef + npts + p, fma(-alpha, ax, beta));
    stv<TS, TC>(coef + 2 * npts + p, fma(alpha, ay, beta));
    stv<TS, TC>(coef + 3 * npts + p, fma(-alpha, ay, beta));
  }
}

// b - sum_k c_k w_k (the off-diagonal part of b - A w)
template <typename TS, int DIM>
__device__ __forceinline__ typename Cmp<TS>::T rhs_minus_offdiag(
    const LvIdx& q, const TS* __restrict__ w, const Coef4<typename Cmp<TS>::T>& c,
    typename Cmp<TS>::T b) {
  typename Cmp<TS>::T t = b;
  t = fma(-c.e, ldv(w + q.e), t);
  t = fma(-c.w, ldv(w + q.w), t);
  if (DIM == 2) {
    t = fma(-c.n, ldv(w + q.n), t);
    t = fma(-c.s, ldv(w + q.s), t);
  }
  return t;
}

// Level constants of A, formed on the host (a uniform division per thread
// costs more FP64 issue slots than the whole 5-point update).
struct MGConst {
  double alpha;  // cadv / (2h)
  double beta;   // -cdiff / h^2
  double D;      // sigma + 2 dim cdiff / h^2 (Jacobi diagonal)
  double dinv;   // omega / D
  double keep;   // 1 - omega
};

MGConst mg_const(const MGLevelDesc& lv, int dim, double sigma, double cadv, double cdiff,
                 double omega) {
  MGConst c;
  const double invh2 = 1.0 / (lv.h * lv.h);
  c.alpha = cadv * 0.5 / lv.h;
  c.beta = -cdiff * invh2;
  c.D = sigma + cdiff * (2 * dim) * invh2;
  c.dinv = omega / c.D;
  c.keep = 1.0 - omega;
  return c;
}

template <typename TS>
__device__ __forceinline__ typename Cmp<TS>::T round_to_storage(typename Cmp<TS>::T v) {
  return (typename Cmp<TS>::T)(TS)v;
}
template <>
__device__ __forceinline__ float round_to_storage<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// Fine-level right-hand side of a reduced-precision V-cycle read straight
// from the FP64 input (b64), rounded to the storage type as a stored copy
// would be; FP64 storage reads its input in place and never takes b64.
template <typename TS>
__device__ __forceinline__ typename Cmp<TS>::T ld_rhs(const TS* b, const double* b64, long long i) {
  typedef typename Cmp<TS>::T TC;
  if (!std::is_same<TS, double>::value && b64) return round_to_storage<TS>((TC)b64[i]);
  return ldv(b + i);
}

// epi_out: also write epi_out = epi_bcoef epi_base + epi_coef w pointwise
// (the mass-only coupling row of L_P, fused into the last sweep).
// WIDE (reduced-precision storage, finest level): read b from the FP64 input
// b64 and write the result to the FP64 output out64 instead of w_out, both
// rounded as the stored copies would be.
template <typename TS, int DIM, int KIND, bool WIDE = false, typename TV = TS>
__global__ void __launch_bounds__(256) k_mg_smooth(MGLevelDesc lv, int ncomp, MGConst k,
                                                   const TV* __restrict__ vel,
                                                   const TS* __restrict__ b,
                                                   const TS* __restrict__ w_in,
                                                   TS* __restrict__ w_out, int first,
                                                   double* __restrict__ epi_out,
                                                   const double* __restrict__ epi_base,
                                                   double epi_coef, double epi_bcoef,
                                                   const double* __restrict__ b64,
                                                   double* __restrict__ out64) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  const TC alpha = TC(k.alpha), beta = TC(k.beta);
  const TC dinv = TC(k.dinv), keep = TC(k.keep);
  auto rhs = [&](long long i) -> TC {
    return WIDE ? round_to_storage<TS>((TC)b64[i]) : ldv(b + i);
  };
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < lv.npts; p += gridDim.x * blockDim.x) {
    const LvIdx q = lv_nbr<DIM>(lv, p);
    if (first) {
      for (int c = 0; c < ncomp; ++c) {
        const long long off = (long long)c * lv.npts;
        const TC v = dinv * rhs(off + p);
        if (WIDE) out64[off + p] = (double)round_to_storage<TS>(v);
        else stv<TS, TC>(w_out + off + p, v);
      }
      continue;
    }
    const Coef4<TC> cf = stencil_coef<TS, DIM, KIND, TV>(q, vel, lv.npts, alpha, beta);
    for (int c = 0; c < ncomp; ++c) {
      const long long off = (long long)c * lv.npts;
      const TC t = rhs_minus_offdiag<TS, DIM>(q, w_in + off, cf, rhs(off + p));
      // w + omega/D (b - D w - sum c w) = (1 - omega) w + omega/D (b - sum c w)
      const TC v = fma(dinv, t, keep * ldv(w_in + off + p));
      const double vo = (double)round_to_storage<TS>(v);
      if (WIDE) out64[off + p] = vo;
      else stv<TS, TC>(w_out + off + p, v);
      if (epi_out) epi_out[off + p] = fma(epi_coef, vo, epi_bcoef * epi_base[off + p]);
    }
  }
}

template <typename TS, int DIM, int KIND, typename TV = TS>
__global__ void __launch_bounds__(256) k_mg_residual(MGLevelDesc lv, int ncomp, MGConst k,
                                                     const TV* __restrict__ vel,
                                                     const TS* __restrict__ b,
                                                     const TS* __restrict__ w, TS* __restrict__ r) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  const TC D = TC(k.D);
  const TC alpha = TC(k.alpha), beta = TC(k.beta);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < lv.npts; p += gridDim.x * blockDim.x) {
    const LvIdx q = lv_nbr<DIM>(lv, p);
    const Coef4<TC> cf = stencil_coef<TS, DIM, KIND, TV>(q, vel, lv.npts, alpha, beta);
    for (int c = 0; c < ncomp; ++c) {
      const long long off = (long long)c * lv.npts;
      const TC t = rhs_minus_offdiag<TS, DIM>(q, w + off, cf, ldv(b + off + p));
      stv<TS, TC>(r + off + p, fma(-D, ldv(w + off + p), t));
    }
  }
}

// Residual after one damped-Jacobi sweep from w = 0, without storing that
// sweep: w = dinv b, so r = b - A w = (1 - omega) b - dinv sum_k c_k b_k.
// The prolongation then rebuilds w = dinv b + P e (k_mg_prolong<SET>).
template <typename TS, int DIM, int KIND, typename TV = TS>
__global__ void __launch_bounds__(256) k_mg_residual0(MGLevelDesc lv, int ncomp, MGConst k,
                                                      const TV* __restrict__ vel,
                                                      const TS* __restrict__ b, TS* __restrict__ r,
                                                      const double* __restrict__ b64) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  const TC alpha = TC(k.alpha), beta = TC(k.beta);
  const TC dinv = TC(k.dinv), keep = TC(k.keep);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < lv.npts; p += gridDim.x * blockDim.x) {
    const LvIdx q = lv_nbr<DIM>(lv, p);
    const Coef4<TC> cf = stencil_coef<TS, DIM, KIND, TV>(q, vel, lv.npts, alpha, beta);
#pragma unroll 1
    for (int c = 0; c < ncomp; ++c) {
      const long long off = (long long)c * lv.npts;
      const TS* bb = b + off;
      const double* bb64 = b64 ? b64 + off : nullptr;
      TC sum = cf.e * ld_rhs(bb, bb64, q.e);
      sum = fma(cf.w, ld_rhs(bb, bb64, q.w), sum);
      if (DIM == 2) {
        sum = fma(cf.n, ld_rhs(bb, bb64, q.n), sum);
        sum = fma(cf.s, ld_rhs(bb, bb64, q.s), sum);
      }
      stv<TS, TC>(r + off + p, fma(-dinv, sum, keep * ld_rhs(bb, bb64, p)));
    }
  }
}

// Two damped-Jacobi sweeps in one launch (2D, temporal blocking): a 32 x 8
// tile loads w_in on its halo-2 window into shared memory, computes the first
// sweep on the halo-1 window (340 points, 11 warp passes against 8 for the
// tile) and the second on the tile.  The intermediate sweep is rounded to the
// storage type, so the result equals two single sweeps bit for bit.  Halves
// the launches and the passes over w; used where a level is latency- or
// memory-bound (coarse levels, FP32/BF16 storage), not on FP64 levels large
// enough to be FP64-issue-bound, where the extra 19% of work would show.
constexpr int kTX = 32, kTY = 8;


// CHEB: Chebyshev acceleration of undamped Jacobi (k.keep = 0): each sweep
// becomes x_new = x_prev + omega (J(x) - x_prev), with x_prev the iterate
// before x; the pair reads x_{k-1} (w_prev) and x_k (w_in) and writes x_{k+1}
// (w_mid) and x_{k+2} (w_out).  `first`: x_0 = 0 (then w_in, w_prev unused).
template <typename TS, int KIND, bool CHEB, typename TV = TS, bool ZK = false>
__global__ void __launch_bounds__(kTX * kTY) k_mg_smooth2(MGLevelDesc lv, int ncomp, MGConst k,
                                                        const TV* __restrict__ vel,
                                                        const TS* __restrict__ b,
                                                        const TS* __restrict__ w_in,
                                                        TS* __restrict__ w_out, int first,
                                                        const TS* __restrict__ w_prev,
                                                        TS* __restrict__ w_mid, double wa64,
                                                        double wb64) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  constexpr int WX = kTX + 2, WY = kTY + 2, NW = WX * WY;  // the halo-1 window
  __shared__ TC s_in[kTY + 4][kTX + 4];
  __shared__ TC s_w1[WY][WX];
  // b, the four off-diagonal coefficients (E, W, N, S) and, for CHEB, x_{k-1}
  // on the halo-1 window, staged with w in one load phase so that both
  // sweeps run out of shared memory
  __shared__ TC s_b[NW];
  __shared__ TC s_c[4][NW];
  __shared__ TC s_p[CHEB ? NW : 1];
  const TC alpha = TC(k.alpha), beta = TC(k.beta), dinv = TC(k.dinv), keep = TC(k.keep);
  const TC wa = TC(wa64), wb = TC(wb64);
  const int n = lv.n, m = n - 1, ln = lv.logn;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  for (int c = blockIdx.z; c < ncomp; c += gridDim.z) {
    const long long off = (long long)c * lv.npts;
    if (!first) {
      for (int q = tid; q < (kTY + 4) * (kTX + 4); q += kTX * kTY) {
        const int ly = q / (kTX + 4), lx = q - ly * (kTX + 4);
        const int gx = (x0 + lx - 2) & m, gy = (y0 + ly - 2) & m;
        s_in[ly][lx] = ldv(w_in + off + tile_pt(gx, gy, ln, n));
      }
    }
    for (int q = tid; q < NW; q += kTX * kTY) {
      const int ly = q / WX, lx = q - ly * WX;
      const int gx = (x0 + lx - 1) & m, gy = (y0 + ly - 1) & m;
      const int gp = tile_pt(gx, gy, ln, n);
      s_b[q] = ldv(b + off + gp);
      TC ce = beta, cw = beta, cn = beta, cs = beta;
      if (KIND == MG_ADVECTIVE) {
        const TC ax = ldv(vel + gp), ay = ldv(vel + lv.npts + gp);
        ce = fma(alpha, ax, beta); cw = fma(-alpha, ax, beta);
        cn = fma(alpha, ay, beta); cs = fma(-alpha, ay, beta);
      } else if (KIND == MG_ADVECTIVE_PRE) {
        ce = ldv(vel + gp); cw = ldv(vel + lv.npts + gp);
        cn = ldv(vel + 2 * lv.npts + gp); cs = ldv(vel + 3 * lv.npts + gp);
      }
      s_c[0][q] = ce; s_c[1][q] = cw; s_c[2][q] = cn; s_c[3][q] = cs;
      if (CHEB) s_p[q] = first ? TC(0) : ldv(w_prev + off + gp);
    }
    __syncthreads();
    // sweep 1 on the halo-1 window
    for (int q = tid; q < NW; q += kTX * kTY) {
      const int ly = q / WX, lx = q - ly * WX;
      TC v;
      if (first) {
        v = dinv * s_b[q];
      } else {
        const int sy = ly + 1, sx = lx + 1;  // position in s_in
        TC t = s_b[q];
        t = fma(-s_c[0][q], s_in[sy][sx + 1], t);
        t = fma(-s_c[1][q], s_in[sy][sx - 1], t);
        t = fma(-s_c[2][q], s_in[sy + 1][sx], t);
        t = fma(-s_c[3][q], s_in[sy - 1][sx], t);
        v = ZK ? dinv * t : fma(dinv, t, keep * s_in[sy][sx]);
        if (CHEB) {
          const TC xp = s_p[q];
          v = fma(wa, v - xp, xp);
        }
      }
      v = round_to_storage<TS>(v);
      s_w1[ly][lx] = v;
      if (CHEB && lx >= 1 && lx <= kTX && ly >= 1 && ly <= kTY) {
        const int gx = (x0 + lx - 1) & m, gy = (y0 + ly - 1) & m;
        stv<TS, TC>(w_mid + off + tile_pt(gx, gy, ln, n), v);
      }
    }
    __syncthreads();
    // sweep 2 on the tile
    {
      const int lx = threadIdx.x, ly = threadIdx.y;
      const int gp = tile_pt(x0 + lx, y0 + ly, ln, n);
      const int sy = ly + 1, sx = lx + 1;
      const int q = sy * WX + sx;  // the tile point in the halo-1 window
      TC t = s_b[q];
      t = fma(-s_c[0][q], s_w1[sy][sx + 1], t);
      t = fma(-s_c[1][q], s_w1[sy][sx - 1], t);
      t = fma(-s_c[2][q], s_w1[sy + 1][sx], t);
      t = fma(-s_c[3][q], s_w1[sy - 1][sx], t);
      TC v = ZK ? dinv * t : fma(dinv, t, keep * s_w1[sy][sx]);
      if (CHEB) {
        const TC xp = first ? TC(0) : s_in[sy + 1][sx + 1];  // x_k at this point
        v = fma(wb, v - xp, xp);
      }
      stv<TS, TC>(w_out + off + gp, v);
    }
    __syncthreads();
  }
}

// Three damped-Jacobi sweeps in one launch, for latency-bound levels: a 32 x TY
// tile loads w on its halo-3 window and b and the coefficients on its halo-2
// window, then sweeps the halo-2 window, the halo-1 window and the tile out
// of shared memory (TY = 8: 1028 point updates for 768 useful ones; TY = 16:
// 1844 for 1536).  Intermediate sweeps are rounded to the storage type: three
// single sweeps bit for bit.  ZK: undamped sweeps (1 - omega = 0, the
// shift-dominated coarsest levels), w = dinv t without the zero term.
template <typename TS, int KIND, int TY, typename TV = TS, bool ZK = false>
__global__ void __launch_bounds__(kTX * TY) k_mg_smooth3(MGLevelDesc lv, int ncomp, MGConst k,
                                                        const TV* __restrict__ vel,
                                                        const TS* __restrict__ b,
                                                        const TS* __restrict__ w_in,
                                                        TS* __restrict__ w_out, int first) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  constexpr int X3 = kTX + 6, Y3 = TY + 6;  // halo-3 window
  constexpr int X2 = kTX + 4, Y2 = TY + 4;  // halo-2 window (b, coefficients)
  __shared__ TC s_w0[Y3][X3];
  __shared__ TC s_w1[Y2][X2];
  __shared__ TC s_b[Y2 * X2];
  __shared__ TC s_c[4][Y2 * X2];
  const TC alpha = TC(k.alpha), beta = TC(k.beta), dinv = TC(k.dinv), keep = TC(k.keep);
  const int n = lv.n, m = n - 1, ln = lv.logn;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  constexpr int NT = kTX * TY;
  for (int c = blockIdx.z; c < ncomp; c += gridDim.z) {
    const long long off = (long long)c * lv.npts;
    if (!first)
      for (int q = tid; q < Y3 * X3; q += NT) {
        const int ly = q / X3, lx = q - ly * X3;
        const int gx = (x0 + lx - 3) & m, gy = (y0 + ly - 3) & m;
        s_w0[ly][lx] = ldv(w_in + off + tile_pt(gx, gy, ln, n));
      }
    for (int q = tid; q < Y2 * X2; q += NT) {
      const int ly = q / X2, lx = q - ly * X2;
      const int gx = (x0 + lx - 2) & m, gy = (y0 + ly - 2) & m;
      const int gp = tile_pt(gx, gy, ln, n);
      s_b[q] = ldv(b + off + gp);
      TC ce = beta, cw = beta, cn = beta, cs = beta;
      if (KIND == MG_ADVECTIVE) {
        const TC ax = ldv(vel + gp), ay = ldv(vel + lv.npts + gp);
        ce = fma(alpha, ax, beta); cw = fma(-alpha, ax, beta);
        cn = fma(alpha, ay, beta); cs = fma(-alpha, ay, beta);
      } else if (KIND == MG_ADVECTIVE_PRE) {
        ce = ldv(vel + gp); cw = ldv(vel + lv.npts + gp);
        cn = ldv(vel + 2 * lv.npts + gp); cs = ldv(vel + 3 * lv.npts + gp);
      }
      s_c[0][q] = ce; s_c[1][q] = cw; s_c[2][q] = cn; s_c[3][q] = cs;
    }
    __syncthreads();
    // sweep 1 on the halo-2 window: s_w0 (halo 3) -> s_w1 (halo 2)
    for (int q = tid; q < Y2 * X2; q += NT) {
      const int ly = q / X2, lx = q - ly * X2;
      TC v;
      if (first) {
        v = dinv * s_b[q];
      } else {
        const int sy = ly + 1, sx = lx + 1;
        TC t = s_b[q];
        t = fma(-s_c[0][q], s_w0[sy][sx + 1], t);
        t = fma(-s_c[1][q], s_w0[sy][sx - 1], t);
        t = fma(-s_c[2][q], s_w0[sy + 1][sx], t);
        t = fma(-s_c[3][q], s_w0[sy - 1][sx], t);
        v = ZK ? dinv * t : fma(dinv, t, keep * s_w0[sy][sx]);
      }
      s_w1[ly][lx] = round_to_storage<TS>(v);
    }
    __syncthreads();
    // sweep 2 on the halo-1 window: s_w1 -> s_w0 (reused, halo-1 positions)
    for (int q = tid; q < (TY + 2) * (kTX + 2); q += NT) {
      const int ly = q / (kTX + 2), lx = q - ly * (kTX + 2);
      const int sy = ly + 1, sx = lx + 1;  // in the halo-2 window
      const int cq = sy * X2 + sx;
      TC t = s_b[cq];
      t = fma(-s_c[0][cq], s_w1[sy][sx + 1], t);
      t = fma(-s_c[1][cq], s_w1[sy][sx - 1], t);
      t = fma(-s_c[2][cq], s_w1[sy + 1][sx], t);
      t = fma(-s_c[3][cq], s_w1[sy - 1][sx], t);
      s_w0[ly][lx] = round_to_storage<TS>(ZK ? dinv * t : fma(dinv, t, keep * s_w1[sy][sx]));
    }
    __syncthreads();
    // sweep 3 on the tile: s_w0 (halo-1 window at [0..TY+1][0..kTX+1]) -> global
    {
      const int lx = threadIdx.x, ly = threadIdx.y;
      const int sy = ly + 1, sx = lx + 1;  // in the halo-1 window
      const int cq = (ly + 2) * X2 + (lx + 2);
      TC t = s_b[cq];
      t = fma(-s_c[0][cq], s_w0[sy][sx + 1], t);
      t = fma(-s_c[1][cq], s_w0[sy][sx - 1], t);
      t = fma(-s_c[2][cq], s_w0[sy + 1][sx], t);
      t = fma(-s_c[3][cq], s_w0[sy - 1][sx], t);
      stv<TS, TC>(w_out + off + tile_pt(x0 + lx, y0 + ly, ln, n),
                  ZK ? dinv * t : fma(dinv, t, keep * s_w0[sy][sx]));
    }
    __syncthreads();
  }
}

// One red-black Gauss-Seidel sweep (2D, undamped) per launch: red points
// ((x + y) even) are updated from their black neighbours, then black points
// from the new red ones.  A 32 x 8 tile loads w on its halo-2 window, updates
// the red points of the halo-1 window in place (170 of 340) and then the black
// points of the tile (128 of 256), so a sweep costs one update per point plus
// 16% on the halo.  For a consistently ordered 5-point operator one GS sweep
// reduces the error like two Jacobi sweeps (rho_GS = rho_J^2).  first: w = 0.
template <typename TS, int KIND, typename TV = TS>
__global__ void __launch_bounds__(kTX * kTY) k_mg_rbgs(MGLevelDesc lv, int ncomp, MGConst k,
                                                     const TV* __restrict__ vel,
                                                     const TS* __restrict__ b,
                                                     const TS* __restrict__ w_in,
                                                     TS* __restrict__ w_out, int first) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  __shared__ TC s_w[kTY + 4][kTX + 4];
  const TC alpha = TC(k.alpha), beta = TC(k.beta), dinv = TC(k.dinv);
  const int n = lv.n, m = n - 1, ln = lv.logn;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  auto coefs = [&](int gp, TC& ce, TC& cw, TC& cn, TC& cs) {
    ce = cw = cn = cs = beta;
    if (KIND == MG_ADVECTIVE) {
      const TC ax = ldv(vel + gp), ay = ldv(vel + lv.npts + gp);
      ce = fma(alpha, ax, beta); cw = fma(-alpha, ax, beta);
      cn = fma(alpha, ay, beta); cs = fma(-alpha, ay, beta);
    } else if (KIND == MG_ADVECTIVE_PRE) {
      ce = ldv(vel + gp); cw = ldv(vel + lv.npts + gp);
      cn = ldv(vel + 2 * lv.npts + gp); cs = ldv(vel + 3 * lv.npts + gp);
    }
  };
  for (int c = blockIdx.z; c < ncomp; c += gridDim.z) {
    const long long off = (long long)c * lv.npts;
    for (int q = tid; q < (kTY + 4) * (kTX + 4); q += kTX * kTY) {
      const int ly = q / (kTX + 4), lx = q - ly * (kTX + 4);
      const int gx = (x0 + lx - 2) & m, gy = (y0 + ly - 2) & m;
      s_w[ly][lx] = first ? TC(0) : ldv(w_in + off + tile_pt(gx, gy, ln, n));
    }
    __syncthreads();
    // red points of the halo-1 window: window row r (0..kTY+1), 17 per row;
    // x0, y0 are even, so (gx + gy) is even where (lx + ly) is even
    for (int q = tid; q < (kTY + 2) * ((kTX + 2) / 2); q += kTX * kTY) {
      const int r = q / ((kTX + 2) / 2), j = q - r * ((kTX + 2) / 2);
      const int cx = 2 * j + (r & 1);  // window column with cx + r even
      const int sy = r + 1, sx = cx + 1;  // position in s_w
      const int gx = (x0 + cx - 1) & m, gy = (y0 + r - 1) & m;
      const int gp = tile_pt(gx, gy, ln, n);
      TC ce, cw, cn, cs;
      coefs(gp, ce, cw, cn, cs);
      TC t = ldv(b + off + gp);
      t = fma(-ce, s_w[sy][sx + 1], t);
      t = fma(-cw, s_w[sy][sx - 1], t);
      t = fma(-cn, s_w[sy + 1][sx], t);
      t = fma(-cs, s_w[sy - 1][sx], t);
      s_w[sy][sx] = round_to_storage<TS>(dinv * t);
    }
    __syncthreads();
    // black points of the tile: 16 per row
    if (tid < kTY * (kTX / 2)) {
      const int r = tid / (kTX / 2), j = tid - r * (kTX / 2);
      const int cx = 2 * j + ((r + 1) & 1);  // tile column with cx + r odd
      const int sy = r + 2, sx = cx + 2;
      const int gp = tile_pt(x0 + cx, y0 + r, ln, n);
      TC ce, cw, cn, cs;
      coefs(gp, ce, cw, cn, cs);
      TC t = ldv(b + off + gp);
      t = fma(-ce, s_w[sy][sx + 1], t);
      t = fma(-cw, s_w[sy][sx - 1], t);
      t = fma(-cn, s_w[sy + 1][sx], t);
      t = fma(-cs, s_w[sy - 1][sx], t);
      s_w[sy][sx] = round_to_storage<TS>(dinv * t);
    }
    __syncthreads();
    {
      const int lx = threadIdx.x, ly = threadIdx.y;
      stv<TS, TC>(w_out + off + tile_pt(x0 + lx, y0 + ly, ln, n), s_w[ly + 2][lx + 2]);
    }
    __syncthreads();
  }
}

// The bottom of a periodic 2D Poisson V-cycle in one CTA: levels n0 = 32 (or
// 16) down to 8 held in shared memory.  Per level above 8: `pre` damped-Jacobi
// sweeps from zero, residual, full weighting; on 8^2 the exact zero-mean
// solve w = A^+ b with the 64 x 64 pseudo-inverse (pinv, row-major, for
// cdiff = 1); back up: bilinear prolongation and `post` sweeps.  The same
// stencils as the multi-launch kernels (A = -cdiff L_h), one point per
// thread on 32^2.  Replaces about a dozen latency-bound launches and the
// 40-sweep coarsest solve of the deep Poisson cycles.
constexpr int kBotThreads = 1024;

// Level constants of the bottom cycle, formed on the host (a division per
// thread and sweep would cost more FP64 issue than the sweep itself).
struct BottomConst {
  int nl;                // levels n0, n0/2, ..., 8
  int n[4], logn[4], off[4];
  double c[4];           // cdiff / h_l^2
  double dinv[4];        // omega / (4 c_l)
  double keep;           // 1 - omega
  double inv_cdiff;
};

template <typename TS>
__global__ void __launch_bounds__(kBotThreads) k_mg_bottom(BottomConst K, int pre, int post,
                                                          const double* __restrict__ pinv,
                                                          const TS* __restrict__ b_in,
                                                          TS* __restrict__ w_out) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  extern __shared__ unsigned char smem_raw[];
  TC* base = reinterpret_cast<TC*>(smem_raw);
  const int tid = threadIdx.x, nl = K.nl;
  auto W = [&](int l) { return base + K.off[l]; };
  auto T = [&](int l) { return base + K.off[l] + K.n[l] * K.n[l]; };
  auto Bv = [&](int l) { return base + K.off[l] + 2 * K.n[l] * K.n[l]; };
  const int n0 = K.n[0];
  for (int k = tid; k < n0 * n0; k += blockDim.x) Bv(0)[k] = ldv(b_in + k);
  __syncthreads();
  const TC keep = TC(K.keep);
  // one damped-Jacobi sweep on level l: src -> dst (src == nullptr: from zero)
  auto sweep = [&](int l, const TC* src, TC* dst) {
    const int n = K.n[l], ln = K.logn[l], m = n - 1, np = n * n;
    const TC c = TC(K.c[l]), dinv = TC(K.dinv[l]);
    const TC* b = Bv(l);
    for (int k = tid; k < np; k += blockDim.x) {
      if (!src) { dst[k] = dinv * b[k]; continue; }
      const int i = k & m, j = k >> ln;
      const TC sn = src[(j << ln) + ((i + 1) & m)] + src[(j << ln) + ((i - 1) & m)] +
                    src[(((j + 1) & m) << ln) + i] + src[(((j - 1) & m) << ln) + i];
      dst[k] = fma(dinv, fma(c, sn, b[k]), keep * src[k]);
    }
    __syncthreads();
  };
  // `cnt` sweeps on level l ending in W(l); from zero when fromzero
  auto smooth = [&](int l, int cnt, bool fromzero) {
    TC* a = W(l);
    TC* t = T(l);
    const int np = K.n[l] * K.n[l];
    if (fromzero && cnt == 0) {
      for (int k = tid; k < np; k += blockDim.x) a[k] = TC(0);
      __syncthreads();
    }
    for (int sw = 0; sw < cnt; ++sw) {
      if (fromzero && sw == 0) { sweep(l, nullptr, a); continue; }
      sweep(l, a, t);
      for (int k = tid; k < np; k += blockDim.x) a[k] = t[k];
      __syncthreads();
    }
  };
  for (int l = 0; l + 1 < nl; ++l) {
    smooth(l, pre, true);
    // residual r = b - A w into T(l), then full weighting into B(l+1)
    const int n = K.n[l], ln = K.logn[l], m = n - 1, np = n * n;
    const TC c = TC(K.c[l]);
    const TC* w = W(l);
    const TC* b = Bv(l);
    TC* r = T(l);
    for (int k = tid; k < np; k += blockDim.x) {
      const int i = k & m, j = k >> ln;
      const TC sn = w[(j << ln) + ((i + 1) & m)] + w[(j << ln) + ((i - 1) & m)] +
                    w[(((j + 1) & m) << ln) + i] + w[(((j - 1) & m) << ln) + i];
      r[k] = fma(c, fma(TC(-4), w[k], sn), b[k]);
    }
    __syncthreads();
    const int nc = n >> 1, lc = ln - 1;
    TC* bc = Bv(l + 1);
    for (int k = tid; k < nc * nc; k += blockDim.x) {
      const int I = k & (nc - 1), J = k >> lc, i = 2 * I, j = 2 * J;
      const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
      const TC centre = r[(j << ln) + i];
      const TC edges = r[(j << ln) + ip] + r[(j << ln) + im] + r[(jp << ln) + i] + r[(jm << ln) + i];
      const TC corners = r[(jp << ln) + ip] + r[(jp << ln) + im] + r[(jm << ln) + ip] + r[(jm << ln) + im];
      bc[k] = (TC(4) * centre + TC(2) * edges + corners) * TC(0.0625);
    }
    __syncthreads();
  }
  {
    // exact zero-mean solve on 8^2: w = A^+ b (A^+ for cdiff = 1, scaled)
    const int l = nl - 1;
    const TC* b = Bv(l);
    TC* w = W(l);
    if (tid < 64) {
      TC acc = 0;
      for (int q = 0; q < 64; ++q) acc = fma(TC(__ldg(pinv + tid * 64 + q)), b[q], acc);
      w[tid] = acc * TC(K.inv_cdiff);
    }
    __syncthreads();
  }
  for (int l = nl - 2; l >= 0; --l) {
    const int n = K.n[l], nc = n >> 1, mc = nc - 1, lc = K.logn[l] - 1;
    const TC* g = W(l + 1);
    TC* f = W(l);
    for (int k = tid; k < nc * nc; k += blockDim.x) {
      const int I = k & mc, J = k >> lc;
      const int I1 = (I + 1) & mc, J1 = (J + 1) & mc;
      const TC c00 = g[(J << lc) + I], c10 = g[(J << lc) + I1];
      const TC c01 = g[(J1 << lc) + I], c11 = g[(J1 << lc) + I1];
      const int o0 = (2 * J) * n + 2 * I, o1 = o0 + n;
      f[o0] += c00;
      f[o0 + 1] += TC(0.5) * (c00 + c10);
      f[o1] += TC(0.5) * (c00 + c01);
      f[o1 + 1] += TC(0.25) * ((c00 + c10) + (c01 + c11));
    }
    __syncthreads();
    smooth(l, post, false);
  }
  for (int k = tid; k < n0 * n0; k += blockDim.x) stv<TS, TC>(w_out + k, W(0)[k]);
}

// Full weighting: fine -> coarse (coarse n = fine n / 2), all components.
template <typename TS, int DIM>
__global__ void __launch_bounds__(256) k_mg_restrict(MGLevelDesc fine, int ncomp,
                                                     const TS* __restrict__ rf,
                                                     TS* __restrict__ bc) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  const int nc = fine.n >> 1, logc = fine.logn - 1, m = fine.n - 1;
  const int ncpts = (DIM == 1) ? nc : nc * nc;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ncpts; p += gridDim.x * blockDim.x) {
#pragma unroll 1
    for (int c = 0; c < ncomp; ++c) {
      const TS* f = rf + (long long)c * fine.npts;
      TC v;
      if (DIM == 1) {
        const int i = 2 * p;
        v = (ldv(f + ((i - 1) & m)) + TC(2) * ldv(f + i) + ldv(f + ((i + 1) & m))) * TC(0.25);
      } else {
        const int I = p & (nc - 1), J = p >> logc;
        const int i = 2 * I, j = 2 * J;
        const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
        const int lf = fine.logn;
        const TC centre = ldv(f + (j << lf) + i);
        const TC edges = ldv(f + (j << lf) + ip) + ldv(f + (j << lf) + im) +
                         ldv(f + (jp << lf) + i) + ldv(f + (jm << lf) + i);
        const TC corners = ldv(f + (jp << lf) + ip) + ldv(f + (jp << lf) + im) +
                           ldv(f + (jm << lf) + ip) + ldv(f + (jm << lf) + im);
        v = (TC(4) * centre + TC(2) * edges + corners) * TC(0.0625);
      }
      stv<TS, TC>(bc + (long long)c * ncpts + p, v);
    }
  }
}

// The folded pre-sweep's residual (k_mg_residual0) and its full-weighting
// restriction (k_mg_restrict) in one launch, 2D.  A CTA owns a 16 x 8 tile of
// coarse points.  It stages b on the fine window that the 3 x 3 weights and
// the 5-point stencil reach (35 x 19 points per component), forms r on the
// 33 x 17 window that the weights read (1.10x the owned 32 x 16 points),
// rounded to the storage type as a stored r would be, and writes the coarse
// right-hand side.  The operations and their order are those of the two
// kernels, so the result is bit-identical, and r never goes to memory.
constexpr int kRCX = 16, kRCY = 8;

template <typename TS, int KIND, typename TV = TS>
__global__ void __launch_bounds__(256) k_mg_resid0_restrict(MGLevelDesc fine, int ncomp, MGConst k,
                                                            const TV* __restrict__ vel,
                                                            const TS* __restrict__ b,
                                                            const double* __restrict__ b64,
                                                            TS* __restrict__ bc) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  constexpr int BX = 2 * kRCX + 3, BY = 2 * kRCY + 3;  // b window: r window + stencil halo
  constexpr int RX = 2 * kRCX + 1, RY = 2 * kRCY + 1;  // r window: owned points + weight halo
  __shared__ TC s_b[2][BY][BX];
  __shared__ TC s_r[2][RY][RX];
  const TC alpha = TC(k.alpha), beta = TC(k.beta), dinv = TC(k.dinv), keep = TC(k.keep);
  const int n = fine.n, m = n - 1, ln = fine.logn, npts = fine.npts;
  const int nc = n >> 1, logc = ln - 1;
  const int I0 = blockIdx.x * kRCX, J0 = blockIdx.y * kRCY;
  const int fx0 = 2 * I0, fy0 = 2 * J0;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < ncomp * BY * BX; q += nt) {
    const int c = q / (BY * BX), rem = q - c * (BY * BX);
    const int ly = rem / BX, lx = rem - ly * BX;
    const int gp = tile_pt((fx0 - 2 + lx) & m, (fy0 - 2 + ly) & m, ln, n);
    const long long off = (long long)c * npts;
    s_b[IRK_IDX(c, 2)][ly][lx] = ld_rhs(b + off, b64 ? b64 + off : nullptr, gp);
  }
  __syncthreads();
  for (int q = tid; q < RY * RX; q += nt) {
    const int ry = q / RX, rx = q - ry * RX;
    LvIdx pt;
    pt.c = tile_pt((fx0 - 1 + rx) & m, (fy0 - 1 + ry) & m, ln, n);
    pt.e = pt.w = pt.n = pt.s = pt.c;  // the 2D kinds read their coefficients at the point
    const Coef4<TC> cf = stencil_coef<TS, 2, KIND, TV>(pt, vel, npts, alpha, beta);
    const int sy = ry + 1, sx = rx + 1;  // the point in the b window
    for (int c = 0; c < ncomp; ++c) {
      TC sum = cf.e * s_b[c][sy][sx + 1];
      sum = fma(cf.w, s_b[c][sy][sx - 1], sum);
      sum = fma(cf.n, s_b[c][sy + 1][sx], sum);
      sum = fma(cf.s, s_b[c][sy - 1][sx], sum);
      s_r[c][ry][rx] = round_to_storage<TS>(fma(-dinv, sum, keep * s_b[c][sy][sx]));
    }
  }
  __syncthreads();
  for (int q = tid; q < ncomp * kRCY * kRCX; q += nt) {
    const int c = q / (kRCY * kRCX), rem = q - c * (kRCY * kRCX);
    const int cy = rem / kRCX, cx = rem - cy * kRCX;
    const int y = 2 * cy + 1, x = 2 * cx + 1;  // fine point (2I, 2J) in the r window
    const TC centre = s_r[c][y][x];
    const TC edges = s_r[c][y][x + 1] + s_r[c][y][x - 1] + s_r[c][y + 1][x] + s_r[c][y - 1][x];
    const TC corners = s_r[c][y + 1][x + 1] + s_r[c][y + 1][x - 1] + s_r[c][y - 1][x + 1] +
                       s_r[c][y - 1][x - 1];
    const TC v = (TC(4) * centre + TC(2) * edges + corners) * TC(0.0625);
    stv<TS, TC>(bc + (long long)c * nc * nc + tile_pt(I0 + cx, J0 + cy, logc, nc), v);
  }
}

// Bilinear (linear in 1D) interpolation of the coarse correction, added to w.
// One thread per coarse point updates the 2x2 (1D: 2) fine points it owns:
// (2I,2J) += c00, (2I+1,2J) += (c00+c10)/2, (2I,2J+1) += (c00+c01)/2,
// (2I+1,2J+1) += (c00+c10+c01+c11)/4.
template <typename TS, int DIM, bool SET>
__global__ void __launch_bounds__(256) k_mg_prolong_add(MGLevelDesc fine, int ncomp,
                                                        const TS* __restrict__ wc,
                                                        TS* __restrict__ wf,
                                                        const TS* __restrict__ bf, double dinv64,
                                                        const double* __restrict__ b64) {
  pdl_entry();
  // SET: w_f = dinv b_f + P e (the fine iterate was one sweep from zero and
  // was never stored); otherwise w_f += P e
  typedef typename Cmp<TS>::T TC;
  const int nc = fine.n >> 1, logc = fine.logn - 1, mc = nc - 1;
  const int ncpts = (DIM == 1) ? nc : nc * nc;
  const TC half = TC(0.5), quarter = TC(0.25), dinv = TC(dinv64);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ncpts; p += gridDim.x * blockDim.x) {
    for (int c = 0; c < ncomp; ++c) {
      const TS* g = wc + (long long)c * ncpts;
      TS* f = wf + (long long)c * fine.npts;
      const TS* fb = SET ? bf + (long long)c * fine.npts : nullptr;
      const double* fb64 = (SET && b64) ? b64 + (long long)c * fine.npts : nullptr;
      auto base = [&](long long o) -> TC { return SET ? dinv * ld_rhs(fb, fb64, o) : ldv(f + o); };
      if (DIM == 1) {
        const TC c0 = ldv(g + p), c1 = ldv(g + ((p + 1) & mc));
        IRK_CHECK(2 * p + 1, fine.npts);
        stv<TS, TC>(f + 2 * p, base(2 * p) + c0);
        stv<TS, TC>(f + 2 * p + 1, base(2 * p + 1) + half * (c0 + c1));
      } else {
        const int I = p & mc, J = p >> logc;
        const int I1 = (I + 1) & mc, J1 = (J + 1) & mc;
        const TC c00 = ldv(g + p), c10 = ldv(g + (J << logc) + I1);
        const TC c01 = ldv(g + (J1 << logc) + I), c11 = ldv(g + (J1 << logc) + I1);
        const int lf = fine.logn;
        const long long o0 = ((long long)(2 * J) << lf) + 2 * I, o1 = o0 + fine.n;
        IRK_CHECK(o1 + 1, fine.npts);
        stv<TS, TC>(f + o0, base(o0) + c00);
        stv<TS, TC>(f + o0 + 1, base(o0 + 1) + half * (c00 + c10));
        stv<TS, TC>(f + o1, base(o1) + half * (c00 + c01));
        stv<TS, TC>(f + o1 + 1, base(o1 + 1) + quarter * ((c00 + c10) + (c01 + c11)));
      }
    }
  }
}

// Coarsest level in one CTA: w = 0, `sweeps` damped-Jacobi sweeps from shared
// memory.  project_mean removes the constant null mode of a pure Laplacian.
template <typename TS, int DIM, int KIND, typename TV = TS>
__global__ void k_mg_coarse(MGLevelDesc lv, int ncomp, double sigma_, double cadv_, double cdiff_,
                            double omega_, int sweeps, int project_mean,
                            const TV* __restrict__ vel, const TS* __restrict__ b,
                            TS* __restrict__ w) {
  pdl_entry();
  typedef typename Cmp<TS>::T TC;
  extern __shared__ unsigned char smem_raw[];
  TC* sw = reinterpret_cast<TC*>(smem_raw);          // ncomp * npts
  TC* sw2 = sw + ncomp * lv.npts;                    // ncomp * npts
  TC* sb = sw2 + ncomp * lv.npts;                    // ncomp * npts
  TC* sv = sb + ncomp * lv.npts;                     // DIM * npts
  __shared__ TC red[32];
  const TC sigma = sigma_, cadv = cadv_, cdiff = cdiff_, omega = omega_;
  const TC inv2h = TC(0.5 / lv.h), invh2 = TC(1.0 / (lv.h * lv.h));
  const TC dinv = omega / (sigma + cdiff * TC(2 * DIM) * invh2);
  const int tot = ncomp * lv.npts;
  for (int k = threadIdx.x; k < tot; k += blockDim.x) {
    sb[k] = ldv(b + k);
    sw[k] = 0;
  }
  for (int k = threadIdx.x; k < DIM * lv.npts; k += blockDim.x) sv[k] = vel ? ldv(vel + k) : TC(0);
  __syncthreads();
  auto remove_mean = [&](TC* f) {
    for (int c = 0; c < ncomp; ++c) {
      if (threadIdx.x == 0) {
        TC s = 0;
        for (int k = 0; k < lv.npts; ++k) s += f[c * lv.npts + k];
        red[0] = s / TC(lv.npts);
      }
      __syncthreads();
      const TC mean = red[0];
      for (int k = threadIdx.x; k < lv.npts; k += blockDim.x) f[c * lv.npts + k] -= mean;
      __syncthreads();
    }
  };
  if (project_mean) remove_mean(sb);
  for (int it = 0; it < sweeps; ++it) {
    for (int k = threadIdx.x; k < tot; k += blockDim.x) {
      const int c = k / lv.npts, p = k - c * lv.npts;
      const LvIdx q = lv_nbr<DIM>(lv, p);
      const TC* f = sw + c * lv.npts;
      const TC wc = f[q.c], we = f[q.e], ww = f[q.w];
      TC lap, adv = 0;
      if (DIM == 1) {
        lap = (we + ww - TC(2) * wc) * invh2;
        if (KIND == MG_ADVECTIVE) adv = sv[q.c] * (we - ww) * inv2h;
        if (KIND == MG_CONSERVATIVE_1D) adv = (sv[q.e] * we - sv[q.w] * ww) * inv2h;
      } else {
        const TC wn = f[q.n], ws = f[q.s];
        lap = (we + ww + wn + ws - TC(4) * wc) * invh2;
        if (KIND == MG_ADVECTIVE) adv = (sv[q.c] * (we - ww) + sv[lv.npts + q.c] * (wn - ws)) * inv2h;
      }
      const TC aw = sigma * wc + cadv * adv - cdiff * lap;
      sw2[k] = wc + dinv * (sb[k] - aw);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < tot; k += blockDim.x) sw[k] = sw2[k];
    __syncthreads();
  }
  if (project_mean) remove_mean(sw);
  for (int k = threadIdx.x; k < tot; k += blockDim.x) stv<TS, TC>(w + k, sw[k]);
}

template <typename TS>
__global__ void k_convert_in(const double* __restrict__ src, TS* __restrict__ dst, long long n) {
  pdl_entry();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    stv<TS, typename Cmp<TS>::T>(dst + p, (typename Cmp<TS>::T)src[p]);
}

template <typename TS>
__global__ void k_convert_out(const TS* __restrict__ src, double* __restrict__ dst, long long n) {
  pdl_entry();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    dst[p] = (double)ldv(src + p);
}

// ---------------------------------------------------------------------------
// Grid of the pointwise (grid-stride) V-cycle kernels: at most six CTAs of
// 256 threads per SM, the number that stays resident at 40 registers (the
// 48-register prolongation fits five).  Measured against four, five and
// eight per SM and an uncapped grid: within 1-2%, six ahead.
static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 6) b = 152 * 6;
  if (b < 1) b = 1;
  return (int)b;
}

size_t mg_elem_size(int prec) { return prec == IRK_MG_FP64 ? sizeof(double) : sizeof(float); }

// TS: storage of the V-cycle's vectors (iterates, right-hand sides,
// residuals); TV: storage of its operator data (the level velocities).
// IRK_MG_BF16 keeps the vectors in FP32 and stores the velocities in BF16.
#define IRK_DISPATCH_PREC(prec, ...)                                                        \
  do {                                                                                      \
    if ((prec) == IRK_MG_FP64) { typedef double TS; typedef double TV; __VA_ARGS__; }       \
    else if ((prec) == IRK_MG_FP32) { typedef float TS; typedef float TV; __VA_ARGS__; }    \
    else { typedef float TS; typedef __nv_bfloat16 TV; __VA_ARGS__; }                       \
  } while (0)

#define IRK_DISPATCH_DK(dim, kind, ...)                                                  \
  do {                                                                                    \
    if ((dim) == 1) {                                                                     \
      if ((kind) == MG_ADVECTIVE) { constexpr int DIM = 1, KIND = MG_ADVECTIVE; __VA_ARGS__; }   \
      else if ((kind) == MG_CONSERVATIVE_1D) { constexpr int DIM = 1, KIND = MG_CONSERVATIVE_1D; __VA_ARGS__; } \
      else { constexpr int DIM = 1, KIND = MG_DIFFUSION; __VA_ARGS__; }                          \
    } else {                                                                              \
      if ((kind) == MG_ADVECTIVE) { constexpr int DIM = 2, KIND = MG_ADVECTIVE; __VA_ARGS__; }   \
      else if ((kind) == MG_ADVECTIVE_PRE) { constexpr int DIM = 2, KIND = MG_ADVECTIVE_PRE; __VA_ARGS__; } \
      else { constexpr int DIM = 2, KIND = MG_DIFFUSION; __VA_ARGS__; }                          \
    }                                                                                     \
  } while (0)

#define IRK_DISPATCH_DK_VEL(dim, kind, ...)                                                  \
  do {                                                                                    \
    if ((dim) == 1) {                                                                     \
      if ((kind) == MG_ADVECTIVE) { constexpr int DIM = 1, KIND = MG_ADVECTIVE; __VA_ARGS__; }   \
      else if ((kind) == MG_CONSERVATIVE_1D) { constexpr int DIM = 1, KIND = MG_CONSERVATIVE_1D; __VA_ARGS__; } \
      else { constexpr int DIM = 1, KIND = MG_DIFFUSION; __VA_ARGS__; }                          \
    } else {                                                                              \
      if ((kind) == MG_ADVECTIVE) { constexpr int DIM = 2, KIND = MG_ADVECTIVE; __VA_ARGS__; }   \
      else { constexpr int DIM = 2, KIND = MG_DIFFUSION; __VA_ARGS__; }                          \
    }                                                                                     \
  } while (0)

void launch_mg_smooth(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                      double cadv, double cdiff, double omega, const void* vel, const void* b,
                      const void* w_in, void* w_out, int first, cudaStream_t st, double* epi_out,
                      const double* epi_base, double epi_coef, double epi_bcoef,
                      const double* b64, double* out64) {
  const MGConst k = mg_const(lv, dim, sigma, cadv, cdiff, omega);
  // FP64 storage reads and writes in place; the wide form needs both pointers
  const bool wide = (prec != IRK_MG_FP64) && b64 && out64;
  if (prec != IRK_MG_FP64 && !wide) epi_out = nullptr;  // the epilogue reads the FP64 result
  IRK_DISPATCH_PREC(prec, IRK_DISPATCH_DK(dim, kind, {
    if (wide)
      launch_pdl(k_mg_smooth<TS, DIM, KIND, true, TV>, grid_for(lv.npts), 256, 0, st, 
          lv, ncomp, k, (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first, epi_out,
          epi_base, epi_coef, epi_bcoef, b64, out64);
    else
      launch_pdl(k_mg_smooth<TS, DIM, KIND, false, TV>, grid_for(lv.npts), 256, 0, st, 
          lv, ncomp, k, (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first, epi_out,
          epi_base, epi_coef, epi_bcoef, nullptr, nullptr);
  }));
}

// Whether one k_mg_smooth2 launch should replace two k_mg_smooth launches.
// Measured on GB300 with two components (time of the pair / time of two
// single sweeps): up to 512^2 the pair wins at every storage precision
// (0.5-0.94); on 1024^2 it loses (1.02-1.15: the staged tile's shared memory
// costs occupancy on a bandwidth- or FP64-bound level) except for the pair
// that starts from zero (its first sweep reads b only) on FP32/BF16 storage
// or a diffusion operator (0.84-0.87).
// Whether one k_mg_smooth3 launch should replace a pair and a single sweep
// (measured on GB300, two components: 0.5-0.93 up to 512^2 at every storage
// precision and on 1024^2 for FP32/BF16; 1.05-1.12 for FP64 on 1024^2).
bool mg_smooth3_pays(int prec, int dim, const MGLevelDesc& lv) {
  if (dim != 2 || lv.n < kTX) return false;
  return lv.n <= 512 || prec != IRK_MG_FP64;
}

bool mg_smooth2_pays(int prec, int dim, int kind, const MGLevelDesc& lv, int first) {
  if (dim != 2 || lv.n < kTX) return false;  // n a power of two: tiles cover the grid
  if (lv.n <= 512) return true;
  return first && (prec != IRK_MG_FP64 || kind == MG_DIFFUSION);
}

void launch_mg_smooth2(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                       double cadv, double cdiff, double omega, const void* vel, const void* b,
                       const void* w_in, void* w_out, int first, cudaStream_t st) {
  const MGConst k = mg_const(lv, 2, sigma, cadv, cdiff, omega);
  // up to 256^2 one CTA per tile and component: twice the warps on a
  // latency-bound level (the velocity coefficients are then formed per
  // component); larger levels loop over the components in one CTA
  const int zsplit = (lv.n <= 256) ? ncomp : 1;
  const dim3 grid(lv.n / kTX, lv.n / kTY, zsplit), block(kTX, kTY);
  if (k.keep == 0.0) {
    IRK_DISPATCH_PREC(prec, {
      if (kind == MG_ADVECTIVE)
        launch_pdl(k_mg_smooth2<TS, MG_ADVECTIVE, false, TV, true>, grid, block, 0, st, lv, ncomp, k,
                   (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first, nullptr,
                   nullptr, 1.0, 1.0);
      else if (kind == MG_ADVECTIVE_PRE)
        launch_pdl(k_mg_smooth2<TS, MG_ADVECTIVE_PRE, false, TV, true>, grid, block, 0, st, lv,
                   ncomp, k, (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first,
                   nullptr, nullptr, 1.0, 1.0);
      else
        launch_pdl(k_mg_smooth2<TS, MG_DIFFUSION, false, TV, true>, grid, block, 0, st, lv, ncomp, k,
                   (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first, nullptr,
                   nullptr, 1.0, 1.0);
    });
    return;
  }
  IRK_DISPATCH_PREC(prec, {
    if (kind == MG_ADVECTIVE)
      launch_pdl(k_mg_smooth2<TS, MG_ADVECTIVE, false, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)w_in, (TS*)w_out, first, nullptr, nullptr, 1.0, 1.0);
    else if (kind == MG_ADVECTIVE_PRE)
      launch_pdl(k_mg_smooth2<TS, MG_ADVECTIVE_PRE, false, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)w_in, (TS*)w_out, first, nullptr, nullptr, 1.0, 1.0);
    else
      launch_pdl(k_mg_smooth2<TS, MG_DIFFUSION, false, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)w_in, (TS*)w_out, first, nullptr, nullptr, 1.0, 1.0);
  });
}

void launch_mg_rbgs(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                    double cadv, double cdiff, const void* vel, const void* b, const void* w_in,
                    void* w_out, int first, cudaStream_t st) {
  const MGConst k = mg_const(lv, 2, sigma, cadv, cdiff, 1.0);  // undamped: dinv = 1/D
  const int zsplit = (lv.n <= 256) ? ncomp : 1;
  const dim3 grid(lv.n / kTX, lv.n / kTY, zsplit), block(kTX, kTY);
  IRK_DISPATCH_PREC(prec, {
    if (kind == MG_ADVECTIVE)
      launch_pdl(k_mg_rbgs<TS, MG_ADVECTIVE, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)w_in, (TS*)w_out, first);
    else if (kind == MG_ADVECTIVE_PRE)
      launch_pdl(k_mg_rbgs<TS, MG_ADVECTIVE_PRE, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)w_in, (TS*)w_out, first);
    else
      launch_pdl(k_mg_rbgs<TS, MG_DIFFUSION, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)w_in, (TS*)w_out, first);
  });
}

void launch_mg_smooth3(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                       double cadv, double cdiff, double omega, const void* vel, const void* b,
                       const void* w_in, void* w_out, int first, cudaStream_t st, int tile_rows) {
  const MGConst k = mg_const(lv, 2, sigma, cadv, cdiff, omega);
  const int zsplit = (lv.n <= 256) ? ncomp : 1;
  // FP64: 32 x 16 tiles, whose sweeps update 1.20x the tile's points against
  // 1.34x for 32 x 8 (the class got 4-6% faster on the 256^2 level); FP32 and
  // BF16 keep 32 x 8, where twice the CTAs measured slightly ahead
  const bool tall = tile_rows == 16 || (tile_rows == 0 && prec == IRK_MG_FP64);
  const int ty = tall ? 16 : kTY;
  const dim3 grid(lv.n / kTX, lv.n / ty, zsplit), block(kTX, ty);
#define IRK_S3(TY_, ZK_)                                                                          \
  do {                                                                                            \
    if (kind == MG_ADVECTIVE)                                                                     \
      launch_pdl(k_mg_smooth3<TS, MG_ADVECTIVE, TY_, TV, ZK_>, grid, block, 0, st, lv, ncomp, k,  \
          (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first);                      \
    else if (kind == MG_ADVECTIVE_PRE)                                                            \
      launch_pdl(k_mg_smooth3<TS, MG_ADVECTIVE_PRE, TY_, TV, ZK_>, grid, block, 0, st, lv, ncomp, \
          k, (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first);                   \
    else                                                                                          \
      launch_pdl(k_mg_smooth3<TS, MG_DIFFUSION, TY_, TV, ZK_>, grid, block, 0, st, lv, ncomp, k,  \
          (const TV*)vel, (const TS*)b, (const TS*)w_in, (TS*)w_out, first);                      \
  } while (0)
  // undamped sweeps (1 - omega = 0) drop the zero term
  const bool zk = (k.keep == 0.0);
  IRK_DISPATCH_PREC(prec, {
    if (tall && zk) IRK_S3(16, true);
    else if (tall) IRK_S3(16, false);
    else if (zk) IRK_S3(kTY, true);
    else IRK_S3(kTY, false);
  });
#undef IRK_S3
}

void launch_mg_cheb2(int prec, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                     double cadv, double cdiff, const void* vel, const void* b, const void* x_prev,
                     const void* x_cur, void* x_mid, void* x_out, double wa, double wb, int first,
                     cudaStream_t st) {
  const MGConst k = mg_const(lv, 2, sigma, cadv, cdiff, 1.0);  // undamped: keep = 0
  const int zsplit = (lv.n <= 256) ? ncomp : 1;
  const dim3 grid(lv.n / kTX, lv.n / kTY, zsplit), block(kTX, kTY);
  IRK_DISPATCH_PREC(prec, {
    if (kind == MG_ADVECTIVE)
      launch_pdl(k_mg_smooth2<TS, MG_ADVECTIVE, true, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)x_cur, (TS*)x_out, first, (const TS*)x_prev, (TS*)x_mid, wa, wb);
    else if (kind == MG_ADVECTIVE_PRE)
      launch_pdl(k_mg_smooth2<TS, MG_ADVECTIVE_PRE, true, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)x_cur, (TS*)x_out, first, (const TS*)x_prev, (TS*)x_mid, wa, wb);
    else
      launch_pdl(k_mg_smooth2<TS, MG_DIFFUSION, true, TV>, grid, block, 0, st, lv, ncomp, k, (const TV*)vel,
          (const TS*)b, (const TS*)x_cur, (TS*)x_out, first, (const TS*)x_prev, (TS*)x_mid, wa, wb);
  });
}

void launch_mg_residual(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp,
                        double sigma, double cadv, double cdiff, const void* vel, const void* b,
                        const void* w, void* r, cudaStream_t st) {
  const MGConst k = mg_const(lv, dim, sigma, cadv, cdiff, 1.0);
  IRK_DISPATCH_PREC(prec, IRK_DISPATCH_DK(dim, kind, (launch_pdl(k_mg_residual<TS, DIM, KIND, TV>, grid_for(lv.npts), 256, 0, st, 
      lv, ncomp, k, (const TV*)vel, (const TS*)b, (const TS*)w, (TS*)r))));
}

void launch_mg_restrict(int prec, int dim, const MGLevelDesc& fine, int ncomp, const void* rf,
                        void* bc, cudaStream_t st) {
  const long long nc = dim == 1 ? fine.n / 2 : (long long)(fine.n / 2) * (fine.n / 2);
  IRK_DISPATCH_PREC(prec, {
    if (dim == 1)
      launch_pdl(k_mg_restrict<TS, 1>, grid_for(nc), 256, 0, st, fine, ncomp, (const TS*)rf, (TS*)bc);
    else
      launch_pdl(k_mg_restrict<TS, 2>, grid_for(nc), 256, 0, st, fine, ncomp, (const TS*)rf, (TS*)bc);
  });
}

void launch_mg_restrict_vel(int prec, int dim, const MGLevelDesc& fine, int ncomp, const void* vf,
                            void* vc, cudaStream_t st) {
  const long long nc = dim == 1 ? fine.n / 2 : (long long)(fine.n / 2) * (fine.n / 2);
  IRK_DISPATCH_PREC(prec, {
    if (dim == 1)
      launch_pdl(k_mg_restrict<TV, 1>, grid_for(nc), 256, 0, st, fine, ncomp, (const TV*)vf, (TV*)vc);
    else
      launch_pdl(k_mg_restrict<TV, 2>, grid_for(nc), 256, 0, st, fine, ncomp, (const TV*)vf, (TV*)vc);
  });
}

size_t mg_vel_size(int prec) {
  return prec == IRK_MG_FP64 ? sizeof(double) : (prec == IRK_MG_FP32 ? sizeof(float) : 2);
}

void launch_mg_prolong_add(int prec, int dim, const MGLevelDesc& fine, int ncomp, const void* wc,
                           void* wf, cudaStream_t st) {
  const long long nc = dim == 1 ? fine.n / 2 : (long long)(fine.n / 2) * (fine.n / 2);
  IRK_DISPATCH_PREC(prec, {
    if (dim == 1)
      launch_pdl(k_mg_prolong_add<TS, 1, false>, grid_for(nc), 256, 0, st, fine, ncomp, (const TS*)wc,
                                                                   (TS*)wf, nullptr, 0.0, nullptr);
    else
      launch_pdl(k_mg_prolong_add<TS, 2, false>, grid_for(nc), 256, 0, st, fine, ncomp, (const TS*)wc,
                                                                   (TS*)wf, nullptr, 0.0, nullptr);
  });
}

void launch_mg_prolong_set(int prec, int dim, const MGLevelDesc& fine, int ncomp, double sigma,
                           double cadv, double cdiff, double omega, const void* bf, const void* wc,
                           void* wf, cudaStream_t st, const double* b64) {
  const MGConst k = mg_const(fine, dim, sigma, cadv, cdiff, omega);
  if (prec == IRK_MG_FP64) b64 = nullptr;
  const long long nc = dim == 1 ? fine.n / 2 : (long long)(fine.n / 2) * (fine.n / 2);
  IRK_DISPATCH_PREC(prec, {
    if (dim == 1)
      launch_pdl(k_mg_prolong_add<TS, 1, true>, grid_for(nc), 256, 0, st, fine, ncomp, (const TS*)wc,
                                                                  (TS*)wf, (const TS*)bf, k.dinv, b64);
    else
      launch_pdl(k_mg_prolong_add<TS, 2, true>, grid_for(nc), 256, 0, st, fine, ncomp, (const TS*)wc,
                                                                  (TS*)wf, (const TS*)bf, k.dinv, b64);
  });
}

// Velocity and stencil coefficients of the two finest levels in one pass
// (FP64 storage, 2D, velocity = the combined field itself): each coarse point
// writes, for the 2 x 2 fine points it owns, the velocity and the four
// coefficients beta +- alpha a (the values k_velocity and k_mg_coef store),
// and for itself the full-weighted velocity (k_mg_restrict's operation order)
// and its coefficients.  One launch instead of four per row.
__global__ void __launch_bounds__(256) k_mg_setup2(MGLevelDesc fine, const double* __restrict__ combo,
                                                   double* __restrict__ vel0,
                                                   double* __restrict__ coef0,
                                                   double* __restrict__ vel1,
                                                   double* __restrict__ coef1, double a0, double b0,
                                                   double a1, double b1) {
  pdl_entry();
  const int nc = fine.n >> 1, logc = fine.logn - 1, m = fine.n - 1, lf = fine.logn;
  const int ncpts = nc * nc, npts = fine.npts;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ncpts; p += gridDim.x * blockDim.x) {
    const int I = p & (nc - 1), J = p >> logc;
    const int i = 2 * I, j = 2 * J;
    const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const double* f = combo + (long long)c * npts;
      double* v0 = vel0 + (long long)c * npts;
      double* cp0 = coef0 + (long long)(2 * c) * npts;  // (e, w) for x, (n, s) for y
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = IRK_IDX(((j + (q >> 1)) << lf) + i + (q & 1), npts);
        const double a = __ldg(f + o);
        v0[o] = a;
        cp0[o] = fma(a0, a, b0);
        cp0[npts + o] = fma(-a0, a, b0);
      }
      const double centre = __ldg(f + (j << lf) + i);
      const double edges = __ldg(f + (j << lf) + ip) + __ldg(f + (j << lf) + im) +
                           __ldg(f + (jp << lf) + i) + __ldg(f + (jm << lf) + i);
      const double corners = __ldg(f + (jp << lf) + ip) + __ldg(f + (jp << lf) + im) +
                             __ldg(f + (jm << lf) + ip) + __ldg(f + (jm << lf) + im);
      const double v = (4.0 * centre + 2.0 * edges + corners) * 0.0625;
      vel1[(long long)c * ncpts + p] = v;
      coef1[(long long)(2 * c) * ncpts + p] = fma(a1, v, b1);
      coef1[(long long)(2 * c + 1) * ncpts + p] = fma(-a1, v, b1);
    }
  }
}

void launch_mg_setup2(const MGLevelDesc& fine, const MGLevelDesc& coarse, double cadv, double cdiff,
                      const double* combo, void* vel0, void* coef0, void* vel1, void* coef1,
                      cudaStream_t st) {
  const MGConst k0 = mg_const(fine, 2, 0.0, cadv, cdiff, 1.0);
  const MGConst k1 = mg_const(coarse, 2, 0.0, cadv, cdiff, 1.0);
  const long long nc = (long long)(fine.n / 2) * (fine.n / 2);
  launch_pdl(k_mg_setup2, grid_for(nc), 256, 0, st, fine, combo, (double*)vel0, (double*)coef0,
                                            (double*)vel1, (double*)coef1, k0.alpha, k0.beta,
                                            k1.alpha, k1.beta);
}

void launch_mg_coef(int prec, const MGLevelDesc& lv, double cadv, double cdiff, const void* vel,
                    void* coef, cudaStream_t st) {
  const MGConst k = mg_const(lv, 2, 0.0, cadv, cdiff, 1.0);
  // the precomputed-coefficient form serves FP64 storage only
  if (prec != IRK_MG_FP64) return;
  launch_pdl(k_mg_coef<double>, grid_for(lv.npts), 256, 0, st, lv, k.alpha, k.beta, (const double*)vel,
                                                      (double*)coef);
}

void launch_mg_residual0(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp,
                         double sigma, double cadv, double cdiff, double omega, const void* vel,
                         const void* b, void* r, cudaStream_t st, const double* b64) {
  const MGConst k = mg_const(lv, dim, sigma, cadv, cdiff, omega);
  if (prec == IRK_MG_FP64) b64 = nullptr;
  IRK_DISPATCH_PREC(prec, IRK_DISPATCH_DK(dim, kind, (launch_pdl(k_mg_residual0<TS, DIM, KIND, TV>, grid_for(lv.npts), 256, 0, st, 
      lv, ncomp, k, (const TV*)vel, (const TS*)b, (TS*)r, b64))));
}

void launch_mg_resid0_restrict(int prec, int kind, const MGLevelDesc& fine, int ncomp,
                               double sigma, double cadv, double cdiff, double omega,
                               const void* vel, const void* b, void* bc, cudaStream_t st,
                               const double* b64) {
  const MGConst k = mg_const(fine, 2, sigma, cadv, cdiff, omega);
  if (prec == IRK_MG_FP64) b64 = nullptr;
  const dim3 grid((fine.n / 2) / kRCX, (fine.n / 2) / kRCY);
  IRK_DISPATCH_PREC(prec, {
    if (kind == MG_ADVECTIVE)
      launch_pdl(k_mg_resid0_restrict<TS, MG_ADVECTIVE, TV>, grid, 256, 0, st, fine, ncomp, k, (const TV*)vel,
                                                                  (const TS*)b, b64, (TS*)bc);
    else if (kind == MG_ADVECTIVE_PRE)
      launch_pdl(k_mg_resid0_restrict<TS, MG_ADVECTIVE_PRE, TV>, grid, 256, 0, st, 
          fine, ncomp, k, (const TV*)vel, (const TS*)b, b64, (TS*)bc);
    else
      launch_pdl(k_mg_resid0_restrict<TS, MG_DIFFUSION, TV>, grid, 256, 0, st, fine, ncomp, k, (const TV*)vel,
                                                                  (const TS*)b, b64, (TS*)bc);
  });
}

void launch_mg_bottom(int prec, const MGLevelDesc& lv, double cdiff, double omega, int pre,
                      int post, const double* pinv, const void* b, void* w, cudaStream_t st) {
  BottomConst K;
  memset(&K, 0, sizeof(K));
  size_t words = 0;
  for (int n = lv.n, l = 0; n >= 8 && l < 4; n >>= 1, ++l) {
    K.n[l] = n;
    K.logn[l] = lv.logn - l;
    K.off[l] = (int)words;
    const double hl = lv.h * (double)(lv.n / n);
    K.c[l] = cdiff / (hl * hl);
    K.dinv[l] = omega / (4.0 * K.c[l]);
    words += 3 * (size_t)n * n;
    K.nl = l + 1;
  }
  K.keep = 1.0 - omega;
  K.inv_cdiff = 1.0 / cdiff;
  IRK_DISPATCH_PREC(prec, {
    typedef typename Cmp<TS>::T TC;
    launch_pdl(k_mg_bottom<TS>, 1, kBotThreads, sizeof(TC) * words, st, K, pre, post, pinv,
        (const TS*)b, (TS*)w);
  });
}

void launch_mg_coarse(int prec, int dim, int kind, const MGLevelDesc& lv, int ncomp, double sigma,
                      double cadv, double cdiff, double omega, int sweeps, int project_mean,
                      const void* vel, const void* b, void* w, cudaStream_t st) {
  IRK_DISPATCH_PREC(prec, {
    typedef typename Cmp<TS>::T TC;
    const size_t smem = sizeof(TC) * ((size_t)3 * ncomp * lv.npts + (size_t)dim * lv.npts);
    // the one-CTA kernel takes the velocity (MG_ADVECTIVE), never precomputed coefficients
    IRK_DISPATCH_DK_VEL(dim, kind, (launch_pdl(k_mg_coarse<TS, DIM, KIND, TV>, 1, 256, smem, st, 
        lv, ncomp, sigma, cadv, cdiff, omega, sweeps, project_mean, (const TV*)vel,
        (const TS*)b, (TS*)w)));
  });
}

void launch_mg_convert_in(int prec, const double* src, void* dst, long long len, cudaStream_t st) {
  IRK_DISPATCH_PREC(prec, (launch_pdl(k_convert_in<TS>, grid_for(len), 256, 0, st, src, (TS*)dst, len)));
}

void launch_mg_convert_out(int prec, const void* src, double* dst, long long len,
                           cudaStream_t st) {
  IRK_DISPATCH_PREC(prec, (launch_pdl(k_convert_out<TS>, grid_for(len), 256, 0, st, (const TS*)src, dst, len)));
}

}  // namespace irk

IRK_BOUNDS_TU(mg)
