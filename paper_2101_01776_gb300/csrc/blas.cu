// FP64 vector kernels of flexible GMRES (step a8).
//
// Classical Gram-Schmidt applied twice (CGS2): every projection pass reads
// the basis once and produces all j+1 inner products together, so one
// iteration costs three streaming passes over the basis instead of the j+1
// dependent passes of modified Gram-Schmidt.  Reductions are deterministic:
// a fixed grid (a function of the vector length only) writes one partial
// per block and value, and a second kernel sums the partials of each value in
// a fixed order, so a run reproduces itself bit for bit.
#include "irk_internal.h"

namespace irk {

static constexpr int kChunk = 8;  // inner products accumulated per sweep

int blas_blocks(long long L) {
  long long b = (L + IRK_BLAS_THREADS * 4 - 1) / (IRK_BLAS_THREADS * 4);
  if (b > 152 * 2) b = 152 * 2;
  if (b < 1) b = 1;
  return (int)b;
}

// Sum kChunk values over the block; thread 0 writes them to out[0..nv).
__device__ __forceinline__ void block_sum_chunk(double (&v)[kChunk], double* sh, double* out,
                                                int nv) {
#pragma unroll
  for (int k = 0; k < kChunk; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kChunk; ++k) sh[k * 32 + wid] = v[k];
  __syncthreads();
  if (threadIdx.x < nv && threadIdx.x < kChunk) {
    double r = 0.0;
    for (int w = 0; w < nw; ++w) r += sh[threadIdx.x * 32 + w];
    out[threadIdx.x] = r;
  }
}

// partials[blk * nv + k] = sum over this block's elements of V_k . w
__global__ void __launch_bounds__(IRK_BLAS_THREADS)
k_multi_dot(const double* __restrict__ V, long long ldv, int nv, const double* __restrict__ w,
            long long L, double* __restrict__ partials) {
  pdl_entry();
  __shared__ double sh[kChunk * 32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int k0 = 0; k0 < nv; k0 += kChunk) {
    double acc[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) acc[k] = 0.0;
    const int kn = min(kChunk, nv - k0);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L; p += stride) {
      const double wv = w[p];
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        if (k < kn) acc[k] = fma(V[(k0 + k) * ldv + p], wv, acc[k]);
    }
    block_sum_chunk(acc, sh, partials + (long long)blockIdx.x * nv + k0, kn);
  }
}

// Exact-count variants for nv <= 16 (the common Krylov depths): every loop
// unrolls to exactly nv FMAs, with no predicated-off slots in the FP64 pipe.
template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* sh, double* out) {
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

template <int NV>
__global__ void __launch_bounds__(IRK_BLAS_THREADS)
k_multi_dot_n(const double* __restrict__ V, long long ldv, const double* __restrict__ w,
              long long L, double* __restrict__ partials) {
  pdl_entry();
  __shared__ double sh[NV * 8];
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    const double wv = w[p];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = fma(V[k * ldv + p], wv, acc[k]);
  }
  block_sum_n<NV>(acc, sh, partials + (long long)blockIdx.x * NV);
}

template <int NV>
__global__ void __launch_bounds__(IRK_BLAS_THREADS)
k_update_dot_n(const double* __restrict__ V, long long ldv, const double* __restrict__ h,
               double* __restrict__ w, long long L, int with_dots, double* __restrict__ partials) {
  pdl_entry();
  __shared__ double sh[(NV + 1) * 8];
  double hk[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) hk[k] = h[k];
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
    if (with_dots) {
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = fma(v[k], x, acc[k]);
    }
    acc[NV] = fma(x, x, acc[NV]);
  }
  if (with_dots) {
    block_sum_n<NV + 1>(acc, sh, partials + (long long)blockIdx.x * (NV + 1));
  } else {
    double nr[1] = {acc[NV]};
    block_sum_n<1>(nr, sh, partials + (long long)blockIdx.x * (NV + 1) + NV);
  }
}

#define IRK_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

void launch_multi_dot(const double* V, long long ldv, int nv, const double* w, long long L,
                      double* partials, cudaStream_t st) {
  const int nb = blas_blocks(L);
  switch (nv) {
#define IRK_MD(N) case N: launch_pdl(k_multi_dot_n<N>, nb, IRK_BLAS_THREADS, 0, st, V, ldv, w, L, partials); return;
    IRK_NV_CASES(IRK_MD)
#undef IRK_MD
    default: launch_pdl(k_multi_dot, nb, IRK_BLAS_THREADS, 0, st, V, ldv, nv, w, L, partials);
  }
}

// w <- w - sum_k h_k V_k; optionally partials of V_k . w_new (k < nv) and
// ||w_new||^2 (index nv), laid out [blk][nv+1].
__global__ void __launch_bounds__(IRK_BLAS_THREADS)
k_update_dot(const double* __restrict__ V, long long ldv, int nv, const double* __restrict__ h,
             double* __restrict__ w, long long L, int with_dots, double* __restrict__ partials) {
  pdl_entry();
  __shared__ double sh[kChunk * 32];
  __shared__ double hs[128];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = h[k];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  double nrm = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L; p += stride) {
    double acc = w[p];
    for (int k = 0; k < nv; ++k) acc = fma(-hs[k], V[k * ldv + p], acc);
    w[p] = acc;
    nrm = fma(acc, acc, nrm);
  }
  if (!with_dots) {
    double v[kChunk];
    v[0] = nrm;
#pragma unroll
    for (int k = 1; k < kChunk; ++k) v[k] = 0.0;
    block_sum_chunk(v, sh, partials + (long long)blockIdx.x * (nv + 1) + nv, 1);
    return;
  }
  const int nvals = nv + 1;
  for (int k0 = 0; k0 < nvals; k0 += kChunk) {
    double acc[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) acc[k] = 0.0;
    const int kn = min(kChunk, nvals - k0);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L; p += stride) {
      const double wv = w[p];
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        const int kk = k0 + k;
        if (k < kn) acc[k] = fma(kk < nv ? V[kk * ldv + p] : wv, wv, acc[k]);
      }
    }
    block_sum_chunk(acc, sh, partials + (long long)blockIdx.x * nvals + k0, kn);
  }
}

void launch_update_dot(const double* V, long long ldv, int nv, const double* hdev, double* w,
                       long long L, int with_dots, double* partials, cudaStream_t st) {
  const int nb = blas_blocks(L);
  switch (nv) {
#define IRK_UD(N) case N: launch_pdl(k_update_dot_n<N>, nb, IRK_BLAS_THREADS, 0, st, V, ldv, hdev, w, L, with_dots, partials); return;
    IRK_NV_CASES(IRK_UD)
#undef IRK_UD
    default:
      launch_pdl(k_update_dot, nb, IRK_BLAS_THREADS, 0, st, V, ldv, nv, hdev, w, L, with_dots, partials);
  }
}

// out[v] = sum_b partials[b * stride + v] in a fixed order, v < gridDim.x
__global__ void k_reduce(const double* __restrict__ partials, int nblk, int stride,
                         double* __restrict__ out) {
  pdl_entry();
  __shared__ double sh[32];
  const int v = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partials[(long long)b * stride + v];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    out[v] = r;
  }
}

void launch_reduce(const double* partials, int nblk, int stride, int nvals, double* out,
                   cudaStream_t st) {
  launch_pdl(k_reduce, nvals, 256, 0, st, partials, nblk, stride, out);
}

__global__ void k_scale_copy(const double* __restrict__ w, double s, double* __restrict__ v,
                             double* __restrict__ v2, long long L) {
  pdl_entry();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    const double x = w[p] * s;
    v[p] = x;
    if (v2) v2[p] = x;
  }
}

void launch_scale_copy(const double* w, double scale, double* v, double* v2, long long L,
                       cudaStream_t st) {
  launch_pdl(k_scale_copy, blas_blocks(L), IRK_BLAS_THREADS, 0, st, w, scale, v, v2, L);
}

struct Coef64 {
  double y[64];
};

__global__ void k_lincomb(double* __restrict__ x, const double* __restrict__ Z, long long ldz, int k,
                          Coef64 c, long long L) {
  pdl_entry();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x) {
    double acc = x[p];
    for (int j = 0; j < k; ++j) acc = fma(c.y[j], Z[j * ldz + p], acc);
    x[p] = acc;
  }
}

void launch_lincomb(double* x, const double* Z, long long ldz, int k, const double* y,
                    long long L, cudaStream_t st) {
  Coef64 c;
  for (int j = 0; j < k && j < 64; ++j) c.y[j] = y[j];
  launch_pdl(k_lincomb, blas_blocks(L), IRK_BLAS_THREADS, 0, st, x, Z, ldz, k, c, L);
}

__global__ void k_norm2(const double* __restrict__ x, long long L, double* __restrict__ partials) {
  pdl_entry();
  __shared__ double sh[kChunk * 32];
  double v[kChunk];
#pragma unroll
  for (int k = 0; k < kChunk; ++k) v[k] = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x)
    v[0] = fma(x[p], x[p], v[0]);
  block_sum_chunk(v, sh, partials + blockIdx.x, 1);
}

void launch_norm2(const double* x, long long L, double* partials, cudaStream_t st) {
  launch_pdl(k_norm2, blas_blocks(L), IRK_BLAS_THREADS, 0, st, x, L, partials);
}

__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b,
                        long long L) {
  pdl_entry();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L;
       p += (long long)gridDim.x * blockDim.x)
    y[p] = (b == 0.0) ? a * x[p] : fma(a, x[p], b * y[p]);
}

void launch_axpby(double* y, double a, const double* x, double b, long long L, cudaStream_t st) {
  launch_pdl(k_axpby, blas_blocks(L), IRK_BLAS_THREADS, 0, st, y, a, x, b, L);
}

#ifdef IRK_BOUNDS
static __device__ double g_selftest_slot[1];

__global__ void k_bounds_selftest(long long index, long long extent) {
  pdl_entry();
  g_selftest_slot[IRK_IDX(index, extent)] = 1.0;
}

void launch_bounds_selftest(cudaStream_t st) { launch_pdl(k_bounds_selftest, 1, 1, 0, st, 1, 1); }
#endif

}  // namespace irk

IRK_BOUNDS_TU(blas)
