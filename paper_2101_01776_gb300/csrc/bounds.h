// Bounds-checked debug build: compile with -DIRK_BOUNDS (the normal build
// compiles every check away).
//
// IRK_IDX(i, n) is i when 0 <= i < n.  Otherwise the check counts a hit in
// this translation unit's device record, keeps the first hit's source line,
// index and extent, and returns 0, so the access stays inside the buffer and
// the kernel runs to completion.  There is no trap and no assert: the context
// stays usable.  After each call the host collects and clears the records of
// every translation unit (bounds_collect), and irk_step reports the first hit
// as an error.  IRK_CHECK(i, n) checks without using the index.
#pragma once

#include <cuda_runtime.h>

namespace irk {

struct BoundsRecord {
  unsigned int hits;
  int line;
  long long index, extent;
};

}  // namespace irk

#if defined(IRK_BOUNDS) && defined(__CUDACC__)

namespace irk {

// one record per translation unit (internal linkage: no relocatable device code)
static __device__ BoundsRecord g_bounds_record;

__device__ __forceinline__ long long bounds_check(long long i, long long n, int line) {
  if (i >= 0 && i < n) return i;
  if (atomicAdd(&g_bounds_record.hits, 1u) == 0u) {
    g_bounds_record.line = line;
    g_bounds_record.index = i;
    g_bounds_record.extent = n;
  }
  return 0;
}

}  // namespace irk

#define IRK_IDX(i, n) ::irk::bounds_check((long long)(i), (long long)(n), __LINE__)
#define IRK_CHECK(i, n) ((void)IRK_IDX(i, n))

// Host accessor of this translation unit's record: copies it to *out, clears
// it and returns 0, or returns -1 when a CUDA call fails.
#define IRK_BOUNDS_TU(name)                                                          \
  namespace irk {                                                                    \
  int bounds_take_##name(BoundsRecord* out) {                                        \
    const BoundsRecord zero = {0u, 0, 0, 0};                                         \
    if (cudaMemcpyFromSymbol(out, g_bounds_record, sizeof(BoundsRecord)) != cudaSuccess) \
      return -1;                                                                     \
    if (cudaMemcpyToSymbol(g_bounds_record, &zero, sizeof(BoundsRecord)) != cudaSuccess) \
      return -1;                                                                     \
    return 0;                                                                        \
  }                                                                                  \
  }

#elif !defined(IRK_BOUNDS)

#define IRK_IDX(i, n) (i)
#define IRK_CHECK(i, n) ((void)0)
#define IRK_BOUNDS_TU(name)

#endif
