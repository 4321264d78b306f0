// irk_measure_alu_peak: the fused multiply-add throughput of the current GPU,
// measured, as the roofline denominator of the kernels bound by FP64 (or, for
// reduced-precision V-cycles, FP32) arithmetic.
//
// Every thread runs kChains independent FMA recurrences a <- a*x + y with
// x slightly below one, so the values stay near y/(1-x) (no overflow, no
// subnormals) and nothing can be folded away; the grid puts 8 blocks of 256
// threads on every SM.  One FMA counts as two floating-point operations.
#include <algorithm>

#include "irk_internal.h"

namespace irk {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T* out, int iters, T x, T y) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], x, y);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
irk_status probe(cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return IRK_ERR_NO_DEVICE;
  }
  const int blocks = 8 * sms;
  const double threads = (double)blocks * kProbeThreads;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  irk_status rc = IRK_OK;
  if (cudaMalloc(&out, sizeof(T) * blocks * kProbeThreads) != cudaSuccess) {
    cudaGetLastError();
    return IRK_ERR_NOMEM;
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = IRK_ERR_CUDA;
  const T x = (T)0.9999, y = (T)1e-4;
  // calibrate on a short run, then time runs of about 20 ms: best of five
  int iters = 1024;
  double best = 0.0;
  for (int rep = 0; rep < 7 && rc == IRK_OK; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, kProbeThreads, 0, st>>>(out, iters, x, y);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        !(ms > 0.f)) {
      rc = IRK_ERR_CUDA;
      break;
    }
    const double rate = 2.0 * kChains * (double)iters * threads / (ms * 1e-3) / 1e12;
    if (rep == 0) {
      // next runs: about 20 ms each, within int range
      const double want = 20.0 / ms * iters;
      iters = (int)std::min(std::max(want, 1024.0), 1.0e9);
      continue;
    }
    best = std::max(best, rate);
  }
  if (rc == IRK_OK && cudaGetLastError() != cudaSuccess) rc = IRK_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == IRK_OK) *tflops = best;
  return rc;
}

}  // namespace
}  // namespace irk

extern "C" irk_status irk_measure_alu_peak(int precision, void* cuda_stream, double* tflops) {
  if (!tflops || (precision != 0 && precision != 1)) return IRK_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  return precision == 0 ? irk::probe<double>(st, tflops) : irk::probe<float>(st, tflops);
}
