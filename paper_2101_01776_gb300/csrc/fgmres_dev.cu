// Device-resident flexible GMRES (step a8): the Arnoldi bookkeeping runs on
// the GPU so that one restart cycle needs no host round trip.
//
// The iteration index j, the Hessenberg matrix, the Givens rotations and the
// rotated right-hand side live in an FGState block in device memory.  The
// basis kernels read j from there (so one captured kernel serves every j).
// The last block of k_fg_gs2 closes an iteration (Hessenberg column,
// rotations, residual estimate) and ends the loop through the conditional
// handle of a CUDA-graph WHILE node once the block has converged, lost its
// basis, or used m iterations; k_fg_next also bounds the loop independently.
// The arithmetic is the one of the host path (CGS2, Givens, back
// substitution), in FP64.  Outside a graph (the solver's per-kernel timing
// mode launches these kernels one by one) the handle is zero and the loop
// state lives only in the FGState block.
#include <cstdint>
#include <initializer_list>

#include "dev_reduce.cuh"
#include "irk_internal.h"

namespace irk {

// ---------------------------------------------------------------------------
// Inner products / updates with the basis size read from device memory.
template <int NV>
__device__ __forceinline__ void dev_block_sum(double (&v)[NV], double* sh, double* out) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 8 + wid] = v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    double r = 0.0;
    for (int w = 0; w < nw; ++w) r += sh[threadIdx.x * 8 + w];
    out[threadIdx.x] = r;
  }
}

// Generic (nv > 16) forms: chunks of 4 values
__device__ void dev_multi_dot_any(const double* __restrict__ V, long long ldv, int nv,
                                  const double* __restrict__ w, long long L,
                                  double* __restrict__ partials, double* sh) {
  for (int k0 = 0; k0 < nv; k0 += 4) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int kn = min(4, nv - k0);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
         p += (long long)gridDim.x * blockDim.x) {
      const double wv = w[p];
      for (int k = 0; k < kn; ++k) acc[k] = fma(V[(k0 + k) * ldv + p], wv, acc[k]);
    }
    double tmp[4];
    dev_block_sum<4>(acc, sh, tmp);
    if (threadIdx.x < kn) partials[(long long)blockIdx.x * nv + k0 + threadIdx.x] = tmp[threadIdx.x];
  }
}

__device__ void dev_update_dot_any(const double* __restrict__ V, long long ldv, int nv,
                                   const double* __restrict__ h, double* __restrict__ w,
                                   long long L, int with_dots, double* __restrict__ partials,
                                   double* sh) {
  double nrm = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double x = w[p];
    for (int k = 0; k < nv; ++k) x = fma(-h[k], V[k * ldv + p], x);
    w[p] = x;
    nrm = fma(x, x, nrm);
  }
  const int nvals = nv + 1;
  if (with_dots) {
    for (int k0 = 0; k0 < nv; k0 += 4) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      const int kn = min(4, nv - k0);
      for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
           p += (long long)gridDim.x * blockDim.x) {
        const double x = w[p];
        for (int k = 0; k < kn; ++k) acc[k] = fma(V[(k0 + k) * ldv + p], x, acc[k]);
      }
      double tmp[4];
      dev_block_sum<4>(acc, sh, tmp);
      if (threadIdx.x < kn) partials[(long long)blockIdx.x * nvals + k0 + threadIdx.x] = tmp[threadIdx.x];
    }
  }
  double nr[1] = {nrm};
  double tmp[1];
  dev_block_sum<1>(nr, sh, tmp);
  if (threadIdx.x == 0) partials[(long long)blockIdx.x * nvals + nv] = tmp[0];
}

#define IRK_DEV_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

// ---------------------------------------------------------------------------
// Start of a cycle: beta = ||b|| (from its reduced square), g = beta e_1,
// first basis scale 1/beta; an empty or non-finite right-hand side ends the
// loop before it starts.
__global__ void k_fg_init(FGState* s, const double* __restrict__ nrm2, const double* __restrict__ rtol,
                          cudaGraphConditionalHandle cond) {
  pdl_entry();
  const double beta = isfinite(nrm2[0]) ? sqrt(fmax(nrm2[0], 0.0)) : nrm2[0];
  s->j = 0;
  s->k = 0;
  s->its = 0;
  s->stopped = 0;
  s->guard = 0;
  s->ctr1 = 0u;  // last-block counters start every cycle at zero
  s->ctr2 = 0u;
  s->beta = beta;
  s->target = rtol[0] * beta;
  s->res = beta;
  for (int i = 0; i <= IRK_FG_MAXM; ++i) s->g[i] = 0.0;
  s->g[0] = beta;
  if (!(beta > 0.0) || !isfinite(beta)) {
    s->status = isfinite(beta) ? 0 : 2;
    s->inv_scale = 0.0;
    if (cond) cudaGraphSetConditional(cond, 0);
  } else {
    s->status = 0;
    s->inv_scale = 1.0 / beta;
    if (cond) cudaGraphSetConditional(cond, 1);  // (re)open the loop for this cycle
  }
}

// v = w * s->inv_scale written to V_j (j from s) and to prec_in
// (vec: the 16-byte form, two points per access; same arithmetic per point)
__global__ void k_fg_scale(const double* __restrict__ w, const FGState* __restrict__ s,
                           double* __restrict__ V, long long ldv, double* __restrict__ prec_in,
                           long long L, int vec) {
  pdl_entry();
  const double sc = s->inv_scale;
  IRK_CHECK(s->j, IRK_FG_MAXM + 1);
  double* vj = V + (long long)s->j * ldv;
  const long long S = (long long)gridDim.x * blockDim.x;
  if (vec) {
    const double2* __restrict__ w2 = reinterpret_cast<const double2*>(w);
    double2* __restrict__ v2 = reinterpret_cast<double2*>(vj);
    double2* __restrict__ p2 = reinterpret_cast<double2*>(prec_in);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (L >> 1); q += S) {
      double2 x = w2[q];
      x.x *= sc;
      x.y *= sc;
      v2[q] = x;
      p2[q] = x;
    }
    return;
  }
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L; p += S) {
    const double x = w[p] * sc;
    vj[p] = x;
    prec_in[p] = x;
  }
}

// y = R^{-1} g on the leading k x k triangle
__global__ void k_fg_solve(FGState* s) {
  pdl_entry();
  const int k = s->k;
  IRK_CHECK(k, IRK_FG_MAXM + 1);
  for (int i = k - 1; i >= 0; --i) {
    double acc = s->g[i];
    for (int q = i + 1; q < k; ++q) acc -= s->H[q * (IRK_FG_MAXM + 1) + i] * s->y[q];
    s->y[i] = acc / s->H[i * (IRK_FG_MAXM + 1) + i];
  }
}

// x += sum_{j<k} y_j Z_j (vec: the 16-byte form; the same order over j per point)
__global__ void k_fg_lincomb(double* __restrict__ x, const double* __restrict__ Z, long long ldz,
                             const FGState* __restrict__ s, long long L, int vec) {
  pdl_entry();
  __shared__ double ys[IRK_FG_MAXM];
  const int k = s->k;
  IRK_CHECK(k, IRK_FG_MAXM + 1);
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = s->y[j];
  __syncthreads();
  const long long S = (long long)gridDim.x * blockDim.x;
  if (vec) {
    const double2* __restrict__ Z2 = reinterpret_cast<const double2*>(Z);
    double2* __restrict__ x2 = reinterpret_cast<double2*>(x);
    const long long ld2 = ldz >> 1;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (L >> 1); q += S) {
      double2 acc = x2[q];
#pragma unroll 4
      for (int j = 0; j < k; ++j) {
        const double2 z = Z2[j * ld2 + q];
        acc.x = fma(ys[j], z.x, acc.x);
        acc.y = fma(ys[j], z.y, acc.y);
      }
      x2[q] = acc;
    }
    return;
  }
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L; p += S) {
    double acc = x[p];
#pragma unroll 4
    for (int j = 0; j < k; ++j) acc = fma(ys[j], Z[j * ldz + p], acc);
    x[p] = acc;
  }
}

// ---------------------------------------------------------------------------
// Fused CGS2 (one Krylov iteration in three kernels).  Each kernel writes one
// partial per block and value; the block that finishes last (atomic counter,
// reset after use) sums the partials in a fixed order, so the results do not
// depend on block scheduling.  The second projection's update is not stored:
// ||w''||^2 = ||w'||^2 - ||h2||^2 (V orthonormal) gives the new Hessenberg
// entry, and w'' = w' - V h2 is formed inside the normalisation kernel.

// The last-block reductions (last_block_reduce, arrive_last) are in
// dev_reduce.cuh.  Every partial of a block here is stored by threads of
// warp 0 (fewer than 32 values, or chunks of 4), so warp 0 alone fences.

// 16-byte form of the first projection: two consecutive points per load and U
// such pairs per thread and pass, so that a warp keeps (nv + 1) U loads of 16
// bytes in flight (U = 2 up to four basis vectors, 1 up to eight; the scalar
// form below otherwise).  Used when L and ldv are even and every vector starts
// on 16 bytes (the launcher checks).  Out-of-range pairs of the last pass load
// zeros, which add nothing to the sums.  (The same form measured slower for
// the update kernels k_fg_gs2 and k_fg_next, which keep the scalar bodies.)
template <int NV>
struct PairsPerPass {
  static constexpr int U = NV <= 4 ? 2 : 1;
};

template <int NV, int U>
__device__ __forceinline__ void gs1_body2(const double* __restrict__ V, long long ldv,
                                          const double* __restrict__ w, long long L,
                                          double* __restrict__ partials, double* sh) {
  const double2* __restrict__ V2 = reinterpret_cast<const double2*>(V);
  const double2* __restrict__ w2 = reinterpret_cast<const double2*>(w);
  const long long L2 = L >> 1, ld2 = ldv >> 1, S = (long long)gridDim.x * blockDim.x;
  const double2 zero = make_double2(0.0, 0.0);
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < L2; q += U * S) {
    double2 wv[U], v[NV][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long qu = q + u * S;
      const bool in = qu < L2;
      wv[u] = in ? w2[qu] : zero;
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k][u] = in ? V2[k * ld2 + qu] : zero;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        acc[k] = fma(v[k][u].x, wv[u].x, acc[k]);
        acc[k] = fma(v[k][u].y, wv[u].y, acc[k]);
      }
  }
  dev_block_sum<NV>(acc, sh, partials + (long long)blockIdx.x * NV);
}

template <int NV>
__device__ __forceinline__ void gs1_body(const double* __restrict__ V, long long ldv,
                                         const double* __restrict__ w, long long L,
                                         double* __restrict__ partials, double* sh) {
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    const double wv = w[p];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = fma(V[k * ldv + p], wv, acc[k]);
  }
  dev_block_sum<NV>(acc, sh, partials + (long long)blockIdx.x * NV);
}

__global__ void __launch_bounds__(IRK_BLAS_THREADS)
k_fg_gs1(const double* __restrict__ V, long long ldv, FGState* s, const double* __restrict__ w,
         long long L, double* __restrict__ partials, double* __restrict__ h1, int vec) {
  pdl_entry();
  __shared__ double sh[17 * 8];
  const int nv = s->j + 1;
  IRK_CHECK(s->j, IRK_FG_MAXM);
  switch (nv) {
#define IRK_C(N)                                                                   \
  case N:                                                                          \
    if constexpr (N <= 8) {                                                        \
      if (vec) {                                                                   \
        gs1_body2<N, PairsPerPass<N>::U>(V, ldv, w, L, partials, sh);              \
        break;                                                                     \
      }                                                                            \
    }                                                                              \
    gs1_body<N>(V, ldv, w, L, partials, sh);                                       \
    break;
    IRK_DEV_NV_CASES(IRK_C)
#undef IRK_C
    default: dev_multi_dot_any(V, ldv, nv, w, L, partials, sh);
  }
  if (arrive_last(&s->ctr1, 32)) {
    last_block_reduce(partials, gridDim.x, nv, nv, h1);
    if (threadIdx.x == 0) s->ctr1 = 0u;
  }
}

// Arnoldi/Givens step of iteration j from h1, h2 (= h2[0..nv)) and ||w'||^2 =
// h2[nv], run by the whole last block of k_fg_gs2.  The operands (h1, the
// rotations so far, g_j) are staged in shared memory by many threads first,
// so that the serial recurrence of thread 0 waits on no global-memory round
// trip; the new column and rotation are stored back the same way.
struct ArnoldiShared {
  double hc[IRK_FG_MAXM + 2];  // column j of the Hessenberg matrix
  double h2[IRK_FG_MAXM + 2];  // second projection and ||w'||^2
  double cs[IRK_FG_MAXM], sn[IRK_FG_MAXM];
  double g[2];                 // g_j, g_{j+1}
};

__device__ void arnoldi_step(FGState* s, const double* __restrict__ h1, ArnoldiShared& A, int m,
                             int maxit, double* its_total, cudaGraphConditionalHandle cond) {
  const int j = s->j;
  const int nv = j + 1;
  IRK_CHECK(j, m);
  IRK_CHECK(m - 1, IRK_FG_MAXM);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    A.hc[i] = __ldcg(h1 + i) + A.h2[i];
    if (i < j) {
      A.cs[i] = s->cs[i];
      A.sn[i] = s->sn[i];
    }
  }
  if (threadIdx.x == 0) A.g[0] = s->g[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    double h2sq = 0.0;
    for (int i = 0; i <= j; ++i) h2sq = fma(A.h2[i], A.h2[i], h2sq);
    const double rem = A.h2[nv] - h2sq;
    const double hn = rem > 0.0 ? sqrt(rem) : 0.0;
    // previous rotations applied to the new column, top to bottom
    double lo = A.hc[0];
    for (int i = 0; i < j; ++i) {
      const double c = A.cs[i], sg = A.sn[i], hi = A.hc[i + 1];
      A.hc[i] = c * lo + sg * hi;
      lo = -sg * lo + c * hi;
    }
    const double hjj = lo;
    const double den = hypot(hjj, hn);
    const double cj = den > 0.0 ? hjj / den : 1.0;
    const double sj = den > 0.0 ? hn / den : 0.0;
    A.cs[j] = cj;
    A.sn[j] = sj;
    A.hc[j] = den;
    A.hc[j + 1] = 0.0;
    const double gj = A.g[0];
    A.g[1] = -sj * gj;
    A.g[0] = cj * gj;
    const double res = fabs(A.g[1]);
    s->res = res;
    s->its += 1;
    its_total[0] += 1.0;
    const bool finite = isfinite(hn) && isfinite(res) && isfinite(A.h2[nv]);
    if (!finite) {
      s->status = 2;
      its_total[1] = 1.0;
    }
    if (!finite || res <= s->target || hn <= 1e-300 || j + 1 >= m || s->its >= maxit) {
      s->k = finite ? j + 1 : 0;
      s->stopped = 1;
      if (cond) cudaGraphSetConditional(cond, 0);
    } else {
      s->j = j + 1;
      s->inv_scale = 1.0 / hn;
    }
  }
  __syncthreads();
  double* Hc = s->H + j * (IRK_FG_MAXM + 1);
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hc[i] = A.hc[i];
  if (threadIdx.x == 0) {
    s->cs[j] = A.cs[j];
    s->sn[j] = A.sn[j];
    s->g[j] = A.g[0];
    s->g[j + 1] = A.g[1];
  }
}

template <int NV>
__device__ __forceinline__ void gs2_body(const double* __restrict__ V, long long ldv,
                                         const double* __restrict__ h1, double* __restrict__ w,
                                         long long L, double* __restrict__ partials, double* sh) {
  double hk[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) hk[k] = __ldcg(h1 + k);
  double acc[NV + 1];
#pragma unroll
  for (int k = 0; k <= NV; ++k) acc[k] = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double v[NV];
    double x = w[p];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = V[k * ldv + p];
      x = fma(-hk[k], v[k], x);
    }
    w[p] = x;
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = fma(v[k], x, acc[k]);
    acc[NV] = fma(x, x, acc[NV]);
  }
  dev_block_sum<NV + 1>(acc, sh, partials + (long long)blockIdx.x * (NV + 1));
}

__global__ void __launch_bounds__(IRK_BLAS_THREADS)
k_fg_gs2(const double* __restrict__ V, long long ldv, FGState* s, const double* __restrict__ h1,
         double* __restrict__ w, long long L, double* __restrict__ partials, double* __restrict__ h2,
         int m, int maxit, double* its_total, cudaGraphConditionalHandle cond) {
  pdl_entry();
  __shared__ double sh[17 * 8];
  const int nv = s->j + 1;
  IRK_CHECK(s->j, IRK_FG_MAXM);
  switch (nv) {
#define IRK_C(N) case N: gs2_body<N>(V, ldv, h1, w, L, partials, sh); break;
    IRK_DEV_NV_CASES(IRK_C)
#undef IRK_C
    default: dev_update_dot_any(V, ldv, nv, h1, w, L, 1, partials, sh);
  }
  if (arrive_last(&s->ctr2, 32)) {
    __shared__ ArnoldiShared A;
    last_block_reduce(partials, gridDim.x, nv + 1, nv + 1, h2, A.h2);
    if (threadIdx.x == 0) s->ctr2 = 0u;
    __syncthreads();
    arnoldi_step(s, h1, A, m, maxit, its_total, cond);
  }
}

// V_{j+1} = (w' - V h2) * inv_scale, also written to prec_in (skipped once the
// loop has stopped); nv = the new j (the basis size of the finished iteration).
template <int NV>
__device__ __forceinline__ void next_body(const double* __restrict__ V, long long ldv,
                                          const double* __restrict__ h2, double sc,
                                          const double* __restrict__ w, double* __restrict__ vn,
                                          double* __restrict__ prec_in, long long L) {
  double hk[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) hk[k] = h2[k];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double x = w[p];
#pragma unroll
    for (int k = 0; k < NV; ++k) x = fma(-hk[k], V[k * ldv + p], x);
    x *= sc;
    vn[p] = x;
    prec_in[p] = x;
  }
}

__global__ void __launch_bounds__(IRK_BLAS_THREADS)
k_fg_next(const double* __restrict__ V, long long ldv, FGState* s,
          const double* __restrict__ h2, const double* __restrict__ w, double* Vout,
          double* __restrict__ prec_in, long long L, int guard_limit,
          cudaGraphConditionalHandle cond) {
  pdl_entry();
  // independent bound on the loop: whatever the Arnoldi step decided, the
  // body runs at most guard_limit times per cycle
  if (blockIdx.x == 0 && threadIdx.x == 0 && !s->stopped) {
    if (++s->guard >= guard_limit) {
      s->status = 3;
      s->stopped = 1;
      if (cond) cudaGraphSetConditional(cond, 0);
    }
  }
  if (s->stopped) return;
  const int nv = s->j;  // basis size before the new vector
  const double sc = s->inv_scale;
  IRK_CHECK(s->j, IRK_FG_MAXM + 1);
  double* vn = Vout + (long long)s->j * ldv;
  switch (nv) {
#define IRK_C(N) case N: next_body<N>(V, ldv, h2, sc, w, vn, prec_in, L); return;
    IRK_DEV_NV_CASES(IRK_C)
#undef IRK_C
    default:
      for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
           p += (long long)gridDim.x * blockDim.x) {
        double x = w[p];
        for (int k = 0; k < nv; ++k) x = fma(-h2[k], V[k * ldv + p], x);
        x *= sc;
        vn[p] = x;
        prec_in[p] = x;
      }
  }
}

// 1 when the 16-byte forms apply: L and the leading dimension even, every
// vector on a 16-byte boundary.
static int pairs_ok(long long L, long long ld, std::initializer_list<const void*> ptrs) {
  if ((L & 1) || (ld & 1)) return 0;
  for (const void* p : ptrs)
    if (reinterpret_cast<uintptr_t>(p) & 15u) return 0;
  return 1;
}

void launch_fg_gs1(const double* V, long long ldv, FGState* s, const double* w, long long L,
                   double* partials, double* h1, cudaStream_t st) {
  launch_pdl(k_fg_gs1, blas_blocks(L), IRK_BLAS_THREADS, 0, st, V, ldv, s, w, L, partials, h1,
             pairs_ok(L, ldv, {V, w}));
}
void launch_fg_gs2(const double* V, long long ldv, FGState* s, const double* h1, double* w,
                   long long L, double* partials, double* h2, int m, int maxit, double* its_total,
                   cudaGraphConditionalHandle cond, cudaStream_t st) {
  launch_pdl(k_fg_gs2, blas_blocks(L), IRK_BLAS_THREADS, 0, st, V, ldv, s, h1, w, L, partials, h2, m, maxit,
             its_total, cond);
}
void launch_fg_next(const double* V_, long long ldv, FGState* s, const double* h2,
                    const double* w, double* V, double* prec_in, long long L, int guard_limit,
                    cudaGraphConditionalHandle cond, cudaStream_t st) {
  launch_pdl(k_fg_next, blas_blocks(L), IRK_BLAS_THREADS, 0, st, V_, ldv, s, h2, w, V, prec_in, L,
             guard_limit, cond);
}

// ---------------------------------------------------------------------------
// Newton control on the device (whole-step graph).  State nw[]:
//   0 ||F(0)||, 1 ||F||, 2 ||F||/||F(0)||, 3 previous ||F||, 4 updates done,
//   5 status (0 ok, IRK_ERR_NEWTON_DIVERGED, IRK_ERR_NEWTON_MAXIT),
//   6 relative residual of the previous Newton iterate.
// The tests and the forcing term are those of the host loop: stop on a
// non-finite residual, at the tolerance, at the iteration limit, or on growth
// by 1e3; otherwise eta = max(min(krylov_rtol, rel) [1e-3 rel if the last
// update gained less than 2x], 0.2 newton_rtol / rel, 1e-13).
__device__ double forcing_term(double rel, double prev_rel, double fn, double prev, int it,
                               double newton_rtol, double krylov_rtol) {
  double eta = fmin(krylov_rtol, rel);
  if (it > 0 && prev > 0.0 && fn > 0.5 * prev) eta = fmin(eta, 1e-3 * rel);
  // finish: if the observed quadratic rate C = rel/prev_rel^2 (an over-estimate
  // while the linear error dominates) predicts C rel^2 <= newton_rtol/4 for an
  // exact step, solve just tightly enough to land at newton_rtol/2
  if (it > 0 && prev_rel > 0.0 && (rel / (prev_rel * prev_rel)) * rel * rel <= 0.25 * newton_rtol)
    eta = fmin(eta, 0.5 * newton_rtol / rel);
  eta = fmax(eta, 0.2 * newton_rtol / rel);
  return fmax(eta, 1e-13);
}

__global__ void k_newton_first(double* nw, const double* __restrict__ f2, double f2_scale,
                               double* rtol_slot, double newton_rtol, double krylov_rtol,
                               cudaGraphConditionalHandle cond) {
  pdl_entry();
  // f2 is tested before any clamp: fmax(NaN, 0) would read as zero; f2_scale
  // = s when f2 holds one of s equal stage residuals
  const double f0 = isfinite(f2[0]) ? sqrt(fmax(f2_scale * f2[0], 0.0)) : f2[0];
  nw[0] = f0;
  nw[1] = f0;
  nw[2] = f0 > 0.0 ? 1.0 : 0.0;
  nw[3] = f0;
  nw[4] = 0.0;
  nw[5] = 0.0;
  if (!isfinite(f0)) {
    nw[5] = (double)IRK_ERR_NEWTON_DIVERGED;
    if (cond) cudaGraphSetConditional(cond, 0);
  } else if (f0 == 0.0) {
    if (cond) cudaGraphSetConditional(cond, 0);  // k = 0 solves the stage equations
  } else {
    nw[6] = 1.0;
    rtol_slot[0] = forcing_term(1.0, 0.0, f0, f0, 0, newton_rtol, krylov_rtol);
    if (cond) cudaGraphSetConditional(cond, 1);
  }
}

// count = 1 after a Newton update; 0 for the check of a warm-start guess.
__global__ void k_newton_ctl(double* nw, const double* __restrict__ f2, double* rtol_slot,
                             double newton_rtol, int maxit, double krylov_rtol, int count,
                             cudaGraphConditionalHandle cond) {
  pdl_entry();
  if (nw[5] != 0.0) return;  // already failed (non-finite ||F(0)||)
  const double fn = isfinite(f2[0]) ? sqrt(fmax(f2[0], 0.0)) : f2[0];
  const int it = (int)nw[4] + count;
  const double rel = fn / nw[0];
  nw[1] = fn;
  nw[2] = rel;
  nw[4] = (double)it;
  int stop = 1;
  if (!isfinite(fn)) nw[5] = (double)IRK_ERR_NEWTON_DIVERGED;
  else if (rel <= newton_rtol || nw[0] == 0.0) nw[5] = 0.0;
  else if (count == 0 && rel > kGuessLimit) nw[5] = (double)kGuessRejected;  // worse than zero
  else if (it >= maxit) nw[5] = (double)IRK_ERR_NEWTON_MAXIT;
  else if (rel > 1e3) nw[5] = (double)IRK_ERR_NEWTON_DIVERGED;
  else stop = 0;
  if (stop) {
    if (cond) cudaGraphSetConditional(cond, 0);
  } else {
    rtol_slot[0] = forcing_term(rel, count ? nw[6] : 0.0, fn, nw[3], it, newton_rtol, krylov_rtol);
    nw[3] = fn;
    nw[6] = rel;
  }
}

// k = 0 already solves the stage equations when ||F(0)|| = 0; a warm-start
// guess is then replaced by zero stages.
__global__ void k_zero_if_unforced(const double* __restrict__ nw, double* __restrict__ K,
                                   long long len) {
  pdl_entry();
  if (nw[0] != 0.0) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < len;
       p += (long long)gridDim.x * blockDim.x)
    K[p] = 0.0;
}

void launch_zero_if_unforced(const double* nw, double* K, long long len, cudaStream_t st) {
  launch_pdl(k_zero_if_unforced, blas_blocks(len), IRK_BLAS_THREADS, 0, st, nw, K, len);
}

void launch_newton_first(double* nw, const double* f2, double f2_scale, double* rtol_slot,
                         double newton_rtol, double krylov_rtol, cudaGraphConditionalHandle cond,
                         cudaStream_t st) {
  launch_pdl(k_newton_first, 1, 1, 0, st, nw, f2, f2_scale, rtol_slot, newton_rtol, krylov_rtol, cond);
}

void launch_newton_ctl(double* nw, const double* f2, double* rtol_slot, double newton_rtol,
                       int maxit, double krylov_rtol, cudaGraphConditionalHandle cond, int count,
                       cudaStream_t st) {
  launch_pdl(k_newton_ctl, 1, 1, 0, st, nw, f2, rtol_slot, newton_rtol, maxit, krylov_rtol, count, cond);
}

// ---------------------------------------------------------------------------
void launch_fg_init(FGState* s, const double* nrm2, const double* rtol,
                    cudaGraphConditionalHandle cond, cudaStream_t st) {
  launch_pdl(k_fg_init, 1, 1, 0, st, s, nrm2, rtol, cond);
}
void launch_fg_scale(const double* w, const FGState* s, double* V, long long ldv, double* prec_in,
                     long long L, cudaStream_t st) {
  launch_pdl(k_fg_scale, blas_blocks(L), IRK_BLAS_THREADS, 0, st, w, s, V, ldv, prec_in, L,
             pairs_ok(L, ldv, {w, V, prec_in}));
}
void launch_fg_solve(FGState* s, cudaStream_t st) { launch_pdl(k_fg_solve, 1, 1, 0, st, s); }
void launch_fg_lincomb(double* x, const double* Z, long long ldz, const FGState* s, long long L,
                       cudaStream_t st) {
  launch_pdl(k_fg_lincomb, blas_blocks(L), IRK_BLAS_THREADS, 0, st, x, Z, ldz, s, L,
             pairs_ok(L, ldz, {x, Z}));
}

}  // namespace irk

IRK_BOUNDS_TU(fgmres)
