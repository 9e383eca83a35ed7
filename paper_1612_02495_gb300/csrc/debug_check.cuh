// Device-side index checks of the debug build (SWEPT_DEBUG=1).
//
// In the debug build every index the device contexts compute is checked before
// it is used:
//   - window positions, rows and components of the shared-memory tiers;
//   - the ranges a tier or level reads and writes;
//   - edge, strip and band buffer indices;
//   - the state's global coordinates, the counters the persistent kernels wait
//     on, and the adjoint's tape slots.
// A failing check skips its access and records the first failure in a
// device word of its translation unit: check id << 48 | index.  The host reads
// and clears the words with swept_debug_status.  Nothing traps, so a failure
// leaves the context usable.
//
// In the release build (SWEPT_DEBUG=0) every check is the constant true and
// compiles away.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef SWEPT_DEBUG
#define SWEPT_DEBUG 0
#endif

namespace swept {
namespace dbg {

enum Check : int {
  WINDOW = 1,   // window position, row or component
  EDGE = 2,     // edge buffer index
  LEVEL = 3,    // range of a tier / level and its stencil reach
  STATE = 4,    // global coordinate of the state
  STRIP = 5,    // 2D strip buffer index
  BAND = 6,     // 2D band buffer index
  COUNTER = 7,  // counter a persistent kernel waits on
  TAPE = 8,     // adjoint tape slot
  PROBE = 9,    // swept_debug_probe
};

// reads and clears the first-failure word of one translation unit
typedef cudaError_t (*FetchFn)(unsigned long long* word);
// adds a translation unit's reader to the library's list (api.cu)
void register_fetch(FetchFn f);

#if SWEPT_DEBUG
static __device__ unsigned long long g_first_failure;

__device__ __forceinline__ bool ok(bool cond, int id, long long index) {
  if (!cond)
    atomicCAS(&g_first_failure, 0ULL,
              ((unsigned long long)id << 48) | ((unsigned long long)index & 0xffffffffffffULL));
  return cond;
}

static cudaError_t fetch_first_failure(unsigned long long* word) {
  cudaError_t e = cudaMemcpyFromSymbol(word, g_first_failure, sizeof(*word));
  const unsigned long long zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_first_failure, &zero, sizeof(zero));
  return e;
}
static const bool g_fetch_registered = (register_fetch(&fetch_first_failure), true);
#else
__device__ __forceinline__ constexpr bool ok(bool, int, long long) { return true; }
#endif

// window position j of row r, component c, in a window of M points per row
__device__ __forceinline__ bool win(int M, int r, int c, int C, int j) {
  return ok(j >= 0 && j < M && (unsigned)r < 2u && (unsigned)c < (unsigned)C, WINDOW, j);
}
// a tier on [lo, hi) reads [lo - R, hi + R) of a window of M points
__device__ __forceinline__ bool level(int M, int lo, int hi, int R) {
  return ok(lo <= hi && lo - R >= 0 && hi + R <= M, LEVEL, (long long)lo * 65536 + hi);
}
__device__ __forceinline__ bool in_range(int64_t i, int64_t n, int id) { return ok(i >= 0 && i < n, id, i); }

}  // namespace dbg
}  // namespace swept
