// CUDA kernels of the 2D swept decomposition (swept2d.cuh) and the classic
// one-launch-per-step 2D kernel, for the 2D FTCS heat equation
//   T' = fma(Fo, (T_W + T_E) + (T_S + T_N), c1 T),  c1 = 1 - 4 Fo,
// the 2D extension of Eq. HeatDisc, evaluated in this order everywhere.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "debug_check.cuh"
#include "ops.cuh"
#include "swept2d.cuh"

namespace swept2d {

using swept::add_rn;
using swept::fma_rn;
using swept::mul_rn;
namespace dbg = swept::dbg;

template <typename T>
struct Heat2dK {
  T fo, c1;
};

// the 5-point update of window point c (row stride M)
template <typename T>
__device__ __forceinline__ T heat2d_point(const T* c, int M, const Heat2dK<T>& k) {
  const T sx = add_rn(c[-1], c[1]);
  const T sy = add_rn(c[-M], c[M]);
  return fma_rn(k.fo, add_rn(sx, sy), mul_rn(k.c1, c[0]));
}

// q = a / b, r = a - q b for 0 <= a <= 1024, 1 <= b <= 256, from rb, an
// approximation of 1/b in single precision.  (a + 1/2) / b lies at least
// 1/(2b) >= 2^-9 away from an integer, and (a + 1/2) * rb is within a few
// ulp of it (at most 2^-11 absolute for quotients below 1025) when rb is
// within 2 ulp of 1/b, so truncation gives the exact quotient.
__device__ __forceinline__ float recip_small(int b) { return __fdividef(1.0f, (float)b); }
__device__ __forceinline__ void divmod_small(int a, int b, float rb, int& q, int& r) {
  q = (int)(((float)a + 0.5f) * rb);
  r = a - q * b;
}
__device__ __forceinline__ void divmod_small(int a, int b, int& q, int& r) { divmod_small(a, b, recip_small(b), q, r); }

// Device context of one block: the two level rows of its (W + 2R)^2 window in
// shared memory.  Loads and stores spread rows over warps and points of a row
// over lanes; a level spreads its rectangle flat over the block.  COHERENT
// (the persistent kernel): global loads go through L2 (ld.global.cg), since
// other blocks of the same launch wrote what is read.
template <typename T, bool COHERENT = false>
struct Dev2Ctx {
  static constexpr int kR = 1;  // the 5-point heat stencil
  T* sm;
  Geom2 g;
  Heat2dK<T> k;
  T* u;
  const T* s_in;
  T* s_out;
  const T* b_in;
  T* b_out;

  __device__ __forceinline__ T& at(int r, int lx, int ly) { return sm[((int64_t)r * g.M + ly) * g.M + lx]; }
  // a window lies within one period of the grid: -R <= coordinate < n + W + R
  __device__ __forceinline__ static int64_t wrap1(int64_t x, int64_t n) { return x < 0 ? x + n : (x >= n ? x - n : x); }
  __device__ __forceinline__ int64_t gidx(int64_t gx, int64_t gy) const {
    return wrap1(gy, g.ny) * g.nx + wrap1(gx, g.nx);
  }
  template <class F>
  __device__ __forceinline__ void for_grid(int nout, int nin, F&& f) {
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31u), nw = (int)(blockDim.x >> 5);
    for (int o = warp; o < nout; o += nw)
      for (int i = lane; i < nin; i += 32) f(o, i);
  }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  // the loop indices the phases split are < 1024 and the divisors <= 64
  __device__ __forceinline__ void divmod(int a, int b, int& q, int& r) const { divmod_small(a, b, q, r); }
  __device__ __forceinline__ static T ld(const T* p) {
    if constexpr (COHERENT)
      return __ldcg(p);
    else
      return *p;
  }
  // debug build: window position and row, and a global coordinate within one
  // period outside the grid (what wrap1 handles)
  __device__ __forceinline__ bool win(int r, int lx, int ly) const {
    return dbg::win(g.M, r, 0, 1, lx) && dbg::win(g.M, r, 0, 1, ly);
  }
  __device__ __forceinline__ bool coord(int64_t gx, int64_t gy) const {
    return dbg::ok(gx >= -g.nx && gx < 2 * g.nx && gy >= -g.ny && gy < 2 * g.ny, dbg::STATE, gy * g.nx + gx);
  }
  __device__ __forceinline__ void load_u(int r, int lx, int ly, int64_t gx, int64_t gy) {
    if (win(r, lx, ly) && coord(gx, gy)) at(r, lx, ly) = ld(u + gidx(gx, gy));
  }
  __device__ __forceinline__ void store_u(int r, int lx, int ly, int64_t gx, int64_t gy) {
    if (win(r, lx, ly) && coord(gx, gy)) u[gidx(gx, gy)] = at(r, lx, ly);
  }
  __device__ __forceinline__ void load_strip(int r, int lx, int ly, int64_t e) {
    if (win(r, lx, ly) && dbg::in_range(e, g.ntx * g.nty * g.Es, dbg::STRIP)) at(r, lx, ly) = ld(s_in + e);
  }
  __device__ __forceinline__ void store_strip(int r, int lx, int ly, int64_t e) {
    if (win(r, lx, ly) && dbg::in_range(e, g.ntx * g.nty * g.Es, dbg::STRIP)) s_out[e] = at(r, lx, ly);
  }
  __device__ __forceinline__ void load_band(int r, int lx, int ly, int64_t e) {
    if (win(r, lx, ly) && dbg::in_range(e, 2 * g.ntx * g.nty * g.Eb, dbg::BAND)) at(r, lx, ly) = ld(b_in + e);
  }
  __device__ __forceinline__ void store_band(int r, int lx, int ly, int64_t e) {
    if (win(r, lx, ly) && dbg::in_range(e, 2 * g.ntx * g.nty * g.Eb, dbg::BAND)) b_out[e] = at(r, lx, ly);
  }
  // level s on the local rectangle [x0, x1) x [y0, y1): row s & 1 from row
  // (s - 1) & 1.  The rectangle's points are spread flat over the block (point
  // i = y w + x to thread i mod blockDim), so narrow regions (bridges, small
  // corners) still fill whole warps.  A window that holds a mirror wall takes
  // the neighbours of its points through swept::nbr (a block-uniform branch).
  __device__ __forceinline__ void level(int s, int, int x0, int x1, int y0, int y1, int64_t ox, int64_t oy) {
    const int M = g.M;
    const T* in = sm + (int64_t)((s & 1) ^ 1) * M * M;
    T* out = sm + (int64_t)(s & 1) * M * M;
    const int w = x1 - x0, n = w * (y1 - y0);
    const int t = (int)threadIdx.x, nt = (int)blockDim.x;
    const bool in_window = dbg::level(M, x0, x1, kR) && dbg::level(M, y0, y1, kR);
    const int wx = axis_wall(g.bc, g.nx, ox, M), wy = axis_wall(g.bc, g.ny, oy, M);
    if (in_window && t < n) {
      int y, x, dy, dx;
      const float rw = recip_small(w);
      divmod_small(t, w, rw, y, x);
      divmod_small(nt, w, rw, dy, dx);
      if (wx == swept::NO_WALL && wy == swept::NO_WALL) {
        // one 32-bit window offset per point: a step of nt points is dy rows
        // and dx columns, plus a row when the column wraps
        int off = (y0 + y) * M + x0 + x;
        const int step = dy * M + dx, wrap = M - w;
        for (int i = t; i < n; i += nt) {
          out[off] = heat2d_point<T>(in + off, M, k);
          x += dx;
          off += step;
          if (x >= w) {
            x -= w;
            off += wrap;
          }
        }
      } else {
        for (int i = t; i < n; i += nt) {
          const int lx = x0 + x, ly = y0 + y;
          const T* row = in + ly * M;
          const T sx = add_rn(row[swept::nbr(lx, -1, wx)], row[swept::nbr(lx, 1, wx)]);
          const T sy = add_rn(in[swept::nbr(ly, -1, wy) * M + lx], in[swept::nbr(ly, 1, wy) * M + lx]);
          out[ly * M + lx] = fma_rn(k.fo, add_rn(sx, sy), mul_rn(k.c1, row[lx]));
          x += dx;
          y += dy;
          if (x >= w) {
            x -= w;
            ++y;
          }
        }
      }
    }
    __syncthreads();
  }
};

template <typename T>
__global__ void __launch_bounds__(1024) k_pyr2d(Geom2 g, Heat2dK<T> k, T* u, T* s_out, int par, int hh,
                                                 int write_top) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Dev2Ctx<T> cx{reinterpret_cast<T*>(smraw), g, k, u, nullptr, s_out, nullptr, nullptr};
  const int64_t b = blockIdx.x;
  run_pyr(cx, g, b % g.ntx, b / g.ntx, par, hh, write_top != 0);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_bridge2d(Geom2 g, Heat2dK<T> k, T* u, const T* s_in, T* b_out, int par,
                                                    int hh, int write_top) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Dev2Ctx<T> cx{reinterpret_cast<T*>(smraw), g, k, u, s_in, nullptr, nullptr, b_out};
  run_bridge(cx, g, (int64_t)blockIdx.x, par, hh, write_top != 0);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_octa2d(Geom2 g, Heat2dK<T> k, T* u, const T* s_in, T* s_out,
                                                  const T* b_in, int odd, int mode, int hh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Dev2Ctx<T> cx{reinterpret_cast<T*>(smraw), g, k, u, s_in, s_out, b_in, nullptr};
  const int64_t b = blockIdx.x;
  run_octa(cx, g, b % g.ntx, b / g.ntx, odd, mode, hh);
}

// ---------------------------------------------------------------------------
// Persistent 2D swept kernel: the whole launch sequence as one queue of items
// (persist2d_item), claimed in order by resident blocks through an atomic
// counter.  Before running an item, thread 0 waits for the counters its inputs
// come from (persist2d_deps); after it, the block publishes its own
// (persist2d_signal).  An item only waits for items earlier in the queue, which
// were claimed by blocks already resident, so the queue always drains.  A wait
// that exceeds spin_limit polls sets the error word to SWEPT_ETIMEOUT (4) and
// every block returns.
// ---------------------------------------------------------------------------
struct Persist2Ctl {
  int* tile_done;             // T tile counters, -1 before the first pyramid
  int* bridge_done;           // 2T bridge counters, -1 before the first bridge
  unsigned long long* queue;  // next item
  int* error;                 // SWEPT_ETIMEOUT (4) once a wait ran out
  uint32_t spin_limit;
  int64_t start_item;         // the first item claimed (0; > 0 only to exercise the timeout path)
};

__device__ __forceinline__ bool persist2d_wait(const int* flag, int need, const Persist2Ctl& c) {
  for (uint32_t i = 0;; ++i) {
    if (*(volatile const int*)flag >= need) return true;
    if (i >= c.spin_limit || *(volatile const int*)c.error != 0) return false;
    __nanosleep(128);
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_persist2d(Geom2 g, Heat2dK<T> k, T* u, T* s0, T* s1, T* b0, T* b1,
                                                     int64_t n, Persist2Ctl ctl) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int64_t s_item;
  __shared__ int s_ok;
  const int64_t total = persist2d_items(g, n);
  T* S[2] = {s0, s1};
  T* B[2] = {b0, b1};
  for (;;) {
    if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(ctl.queue, 1ULL) + ctl.start_item;
    __syncthreads();
    const int64_t item = s_item;
    if (item >= total) break;
    const PItem it = persist2d_item(g, n, item);
    if (threadIdx.x == 0) {
      bool ok = *(volatile int*)ctl.error == 0;
      int counter[4];
      int64_t index[4], need[4];
      const int nd = persist2d_deps(g, n, it, counter, index, need);
      for (int i = 0; ok && i < nd; ++i)
        ok = dbg::in_range(index[i], (counter[i] ? 2 : 1) * g.ntx * g.nty, dbg::COUNTER) &&
             persist2d_wait((counter[i] ? ctl.bridge_done : ctl.tile_done) + index[i], (int)need[i], ctl);
      if (!ok) atomicCAS(ctl.error, 0, 4);
      s_ok = ok;
      __threadfence();
    }
    __syncthreads();
    if (!s_ok) break;
    const PWork w = persist2d_work(g, n, it);
    Dev2Ctx<T, true> cx{reinterpret_cast<T*>(smraw), g, k, u, S[w.s_in], S[w.s_out], B[w.b_in], B[w.b_out]};
    const int64_t tx = it.idx % g.ntx, ty = it.idx / g.ntx;
    if (it.kind == K_PYR)
      run_pyr(cx, g, tx, ty, w.par, w.hh, w.mode == M2_GAP);
    else if (it.kind == K_BRIDGE)
      run_bridge(cx, g, it.idx, w.par, w.hh, w.mode == M2_GAP);
    else
      run_octa(cx, g, tx, ty, w.par, w.mode, w.hh);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      int sc;
      int64_t si, ss;
      persist2d_signal(g, n, it, &sc, &si, &ss);
      atomicExch((sc ? ctl.bridge_done : ctl.tile_done) + si, (int)ss);
    }
  }
}

// copies a device-side error word into the handle's status word (first error wins)
static __global__ void k_latch_error2d(const int* err, int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *err != 0 && *status == 0) *status = *err;
}

// classic: one step of the whole grid, global memory in and out; periodic
// (bc 0) or mirror walls at -1/2 and n - 1/2 (bc 1: cell -1 reads cell 0, cell
// n reads cell n - 1)
template <typename T>
__global__ void __launch_bounds__(256) k_classic2d(int64_t nx, int64_t ny, int bc, Heat2dK<T> k,
                                                   const T* __restrict__ in, T* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= nx) return;
  const int64_t iw = i == 0 ? (bc ? 0 : nx - 1) : i - 1, ie = i == nx - 1 ? (bc ? nx - 1 : 0) : i + 1;
  const int64_t js = j == 0 ? (bc ? 0 : ny - 1) : j - 1, jn = j == ny - 1 ? (bc ? ny - 1 : 0) : j + 1;
  const T sx = add_rn(in[j * nx + iw], in[j * nx + ie]);
  const T sy = add_rn(in[js * nx + i], in[jn * nx + i]);
  out[j * nx + i] = fma_rn(k.fo, add_rn(sx, sy), mul_rn(k.c1, in[j * nx + i]));
}

}  // namespace swept2d
