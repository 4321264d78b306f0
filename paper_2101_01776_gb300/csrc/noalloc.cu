// irk_stage_residual_noalloc: the stage residual and its 2-norm, computed
// without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a host whose memory manager owns the
// whole device pool and forbids raw allocations, a latency-critical loop in
// which cudaMalloc/cudaFree would synchronise the device and stall other
// streams, or an embedding with a fixed device-memory budget.  This entry
// point therefore takes only caller-owned inputs and outputs and keeps its
// one piece of scratch -- the per-block partial sums of ||F||^2 -- in a
// file-scope device array of fixed size.
//
// It is a variant of the stage-residual kernel: instead of reading stage
// states Y_i from a buffer, each thread forms Y_i = u + dt sum_j a_ij k_j at
// the stencil points it needs, so no Y buffer exists.
#include <cstdio>
#include <mutex>

#include "irk_internal.h"

namespace irk {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 4096;  // 1 partial per block: 32 KiB of scratch

// Shared by every call on a device; holds the last call's partials.
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks];

// Device address of g_noalloc_partials per device (host code may not use the
// symbol itself: on the host it names a stand-in, not device memory).
static void* g_partials_addr[64];
static std::mutex g_partials_mutex;

struct NoallocArgs {
  int n, logn, npts, s;
  double h, inv2h, inv4h, invh2, inv12h2, nu, dt;
  double A[IRK_MAXS * IRK_MAXS];
  const double* u;
  const double* K;
  double* F;
  double* partials;
};

__device__ __forceinline__ int wrap_idx(int i, int n) { return i & (n - 1); }

// Stage state i, component c, at grid point q.
__device__ __forceinline__ double y_at(const NoallocArgs& a, int S, long long L, int i, int c,
                                       int q) {
  double acc = 0.0;
  for (int j = 0; j < S; ++j) acc = fma(a.A[i * S + j], a.K[j * L + (long long)c * a.npts + q], acc);
  return fma(a.dt, acc, a.u[(long long)c * a.npts + q]);
}

// Fill v[dy+1][dx+1] with Y_i (component c) on the 3x3 neighbourhood of (x, y).
__device__ __forceinline__ void y9(const NoallocArgs& a, int S, long long L, int i, int c, int x,
                                   int y, double v[3][3]) {
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int q = IRK_IDX((wrap_idx(y + dy, a.n) << a.logn) + wrap_idx(x + dx, a.n), a.npts);
      v[dy + 1][dx + 1] = y_at(a, S, L, i, c, q);
    }
}

template <int OP, int S>
__global__ void __launch_bounds__(kNoallocThreads) k_residual_noalloc(NoallocArgs a) {
  __shared__ double sh[kNoallocThreads / 32];
  constexpr int C = (OP == IRK_OP_BURGERS_2D || OP == IRK_OP_VSF_2D) ? 2 : 1;
  const long long L = (long long)C * a.npts;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double sq = 0.0;
  if (p < a.npts) {
    for (int i = 0; i < S; ++i) {
      double nv[2] = {0.0, 0.0};
      if (OP == IRK_OP_DIFFUSION_1D || OP == IRK_OP_BURGERS_1D) {
        const double yc = y_at(a, S, L, i, 0, p);
        const double ye = y_at(a, S, L, i, 0, wrap_idx(p + 1, a.n));
        const double yw = y_at(a, S, L, i, 0, wrap_idx(p - 1, a.n));
        nv[0] = a.nu * (ye - 2.0 * yc + yw) * a.invh2;
        if (OP == IRK_OP_BURGERS_1D) nv[0] -= (ye * ye - yw * yw) * a.inv4h;
      } else {
        const int x = p & (a.n - 1), y = p >> a.logn;
        double f0[3][3], f1[3][3];
        y9(a, S, L, i, 0, x, y, f0);
        y9(a, S, L, i, 1, x, y, f1);
        const double l0 = (f0[1][2] + f0[1][0] + f0[2][1] + f0[0][1] - 4.0 * f0[1][1]) * a.invh2;
        const double l1 = (f1[1][2] + f1[1][0] + f1[2][1] + f1[0][1] - 4.0 * f1[1][1]) * a.invh2;
        if (OP == IRK_OP_BURGERS_2D) {
          const double uc = f0[1][1], vc = f1[1][1];
          const double ux = (f0[1][2] - f0[1][0]) * a.inv2h, uy = (f0[2][1] - f0[0][1]) * a.inv2h;
          const double vx = (f1[1][2] - f1[1][0]) * a.inv2h, vy = (f1[2][1] - f1[0][1]) * a.inv2h;
          nv[0] = -uc * ux - vc * uy + a.nu * l0;
          nv[1] = -uc * vx - vc * vy + a.nu * l1;
        } else {  // VSF: f0 = omega, f1 = psi; Arakawa J_A(psi, omega)
          const double (&ps)[3][3] = f1;
          const double (&w)[3][3] = f0;
          const double jpp = (ps[1][2] - ps[1][0]) * (w[2][1] - w[0][1]) -
                             (ps[2][1] - ps[0][1]) * (w[1][2] - w[1][0]);
          const double jpx = ps[1][2] * (w[2][2] - w[0][2]) - ps[1][0] * (w[2][0] - w[0][0]) -
                             ps[2][1] * (w[2][2] - w[2][0]) + ps[0][1] * (w[0][2] - w[0][0]);
          const double jxp = w[2][1] * (ps[2][2] - ps[2][0]) - w[0][1] * (ps[0][2] - ps[0][0]) -
                             w[1][2] * (ps[2][2] - ps[0][2]) + w[1][0] * (ps[2][0] - ps[0][0]);
          nv[0] = (jpp + jpx + jxp) * a.inv12h2 + a.nu * l0;
          nv[1] = -l1 - w[1][1];
        }
      }
      for (int c = 0; c < C; ++c) {
        const double mass = (OP == IRK_OP_VSF_2D && c == 1) ? 0.0 : 1.0;
        const long long idx = i * L + (long long)c * a.npts + p;
        const double f = mass * a.K[idx] - nv[c];
        a.F[idx] = f;
        sq = fma(f, f, sq);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNoallocThreads / 32; ++w) t += sh[w];
    a.partials[blockIdx.x] = t;  // every slot in use is rewritten by this call
  }
}

// ||F||_2 from the partials of this call, summed in a fixed order.
__global__ void __launch_bounds__(kNoallocThreads) k_noalloc_norm(const double* __restrict__ partials,
                                                                  int nblk, double* __restrict__ out) {
  __shared__ double sh[kNoallocThreads / 32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partials[b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNoallocThreads / 32; ++w) t += sh[w];
    *out = sqrt(t);
  }
}

template <int OP>
void launch_noalloc_op(const NoallocArgs& a, int nblk, cudaStream_t st) {
  switch (a.s) {
    case 1: k_residual_noalloc<OP, 1><<<nblk, kNoallocThreads, 0, st>>>(a); break;
    case 2: k_residual_noalloc<OP, 2><<<nblk, kNoallocThreads, 0, st>>>(a); break;
    case 3: k_residual_noalloc<OP, 3><<<nblk, kNoallocThreads, 0, st>>>(a); break;
    case 4: k_residual_noalloc<OP, 4><<<nblk, kNoallocThreads, 0, st>>>(a); break;
    case 5: k_residual_noalloc<OP, 5><<<nblk, kNoallocThreads, 0, st>>>(a); break;
  }
}

}  // namespace
}  // namespace irk

using namespace irk;

extern "C" irk_status irk_stage_residual_noalloc(int op, int n, double length, double nu,
                                                 int stages, const double* A, double dt,
                                                 const double* u, const double* K, double* F,
                                                 double* fnorm, void* cuda_stream) {
  if (op < IRK_OP_DIFFUSION_1D || op > IRK_OP_VSF_2D || stages < 1 || stages > IRK_MAXS ||
      n < 8 || n > 8192 || (n & (n - 1)) || !(length > 0) || !(nu > 0) || !(dt > 0) || !A ||
      !u || !K || !F || !fnorm) {
    fprintf(stderr, "irk_stage_residual_noalloc: invalid argument\n");
    return IRK_ERR_INVALID;
  }
  const int dim = (op == IRK_OP_BURGERS_2D || op == IRK_OP_VSF_2D) ? 2 : 1;
  const long long npts = (dim == 2) ? (long long)n * n : n;
  const long long nblk = (npts + kNoallocThreads - 1) / kNoallocThreads;
  if (nblk > kNoallocMaxBlocks) {
    fprintf(stderr,
            "irk_stage_residual_noalloc: %lld grid points exceed the static scratch "
            "limit of %d points\n",
            npts, kNoallocMaxBlocks * kNoallocThreads);
    return IRK_ERR_NOMEM;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return IRK_ERR_NO_DEVICE;
  }
  // The kernels run on the current device and read and write the four
  // buffers directly: each must be device (or managed) memory of that device.
  // A buffer of another GPU would be reached without peer access, and host
  // memory not at all; both are argument errors, found before any launch.
  {
    const void* bufs[4] = {u, K, F, fnorm};
    const char* names[4] = {"u", "K", "F", "fnorm"};
    for (int b = 0; b < 4; ++b) {
      cudaPointerAttributes attr;
      if (cudaPointerGetAttributes(&attr, bufs[b]) != cudaSuccess ||
          (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
          (attr.type == cudaMemoryTypeDevice && attr.device != dev)) {
        cudaGetLastError();
        fprintf(stderr,
                "irk_stage_residual_noalloc: %s is not device memory of the current device %d\n",
                names[b], dev);
        return IRK_ERR_INVALID;
      }
    }
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_partials_mutex);
    if (!g_partials_addr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_partials_addr[dev], g_noalloc_partials);
      if (e != cudaSuccess) {
        g_partials_addr[dev] = nullptr;
        fprintf(stderr, "irk_stage_residual_noalloc: cudaGetSymbolAddress failed: %s\n",
                cudaGetErrorString(e));
        return IRK_ERR_CUDA;
      }
    }
    scratch = g_partials_addr[dev];
  }
  NoallocArgs a;
  a.n = n;
  a.logn = 0;
  while ((1 << a.logn) < n) ++a.logn;
  a.npts = (int)npts;
  a.s = stages;
  a.h = length / n;
  a.inv2h = 0.5 / a.h;
  a.inv4h = 0.25 / a.h;
  a.invh2 = 1.0 / (a.h * a.h);
  a.inv12h2 = 1.0 / (12.0 * a.h * a.h);
  a.nu = nu;
  a.dt = dt;
  for (int i = 0; i < stages * stages; ++i) a.A[i] = A[i];
  a.u = u;
  a.K = K;
  a.F = F;
  a.partials = (double*)scratch;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  switch (op) {
    case IRK_OP_DIFFUSION_1D: launch_noalloc_op<IRK_OP_DIFFUSION_1D>(a, (int)nblk, st); break;
    case IRK_OP_BURGERS_1D: launch_noalloc_op<IRK_OP_BURGERS_1D>(a, (int)nblk, st); break;
    case IRK_OP_BURGERS_2D: launch_noalloc_op<IRK_OP_BURGERS_2D>(a, (int)nblk, st); break;
    case IRK_OP_VSF_2D: launch_noalloc_op<IRK_OP_VSF_2D>(a, (int)nblk, st); break;
  }
  k_noalloc_norm<<<1, kNoallocThreads, 0, st>>>((const double*)scratch, (int)nblk, fnorm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "irk_stage_residual_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return IRK_ERR_CUDA;
  }
#ifdef IRK_BOUNDS
  {
    // the debug build waits for the kernels and fails the call on any hit
    std::string msg;
    const long long hits = cudaStreamSynchronize(st) == cudaSuccess ? bounds_collect(&msg) : -1;
    if (hits != 0) {
      fprintf(stderr, "irk_stage_residual_noalloc: bounds check: %s\n",
              hits < 0 ? "records could not be read" : msg.c_str());
      return IRK_ERR_CUDA;
    }
  }
#endif
  return IRK_OK;
}

IRK_BOUNDS_TU(noalloc)
