// Deterministic grid reductions by the block that finishes last: every block
// stores one partial per value, counts itself in with an atomic, and the last
// block to arrive sums the partials of all blocks in block order.  The result
// does not depend on the order in which blocks run.  Device code only.
#pragma once

#include <cuda_runtime.h>

namespace irk {

// Sum `count` values (stride `stride`) of the partials of all blocks; called by
// the whole last block; out[v] = sum_b partials[b*stride + v] (in b order),
// also copied to the shared array sout when given.
__device__ __forceinline__ void last_block_reduce(const double* partials, int nblk, int stride,
                                                  int count, double* out, double* sout = nullptr) {
  constexpr int R = 10;  // loads in flight per lane (304 blocks = 9.5 per lane)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = wid; v < count; v += nw) {
    double acc = 0.0;
    for (int b0 = lane; b0 < nblk; b0 += 32 * R) {
      double t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int b = b0 + 32 * r;
        t[r] = b < nblk ? __ldcg(partials + (long long)b * stride + v) : 0.0;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) acc += t[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      out[v] = acc;
      if (sout) sout[v] = acc;
    }
  }
}

// Count this block in; true in the block that arrives last.  The threads
// below `writers` stored this block's partials: their fence publishes them
// before the count (fences are per warp, so a small `writers` keeps the cost
// to one or two warps).
__device__ __forceinline__ bool arrive_last(unsigned int* ctr, int writers) {
  __shared__ bool last;
  if (threadIdx.x < writers) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ctr, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

}  // namespace irk
