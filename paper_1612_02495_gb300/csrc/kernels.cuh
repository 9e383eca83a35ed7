// CUDA kernels: swept passes (up-triangle, diamond, down/gap) and the classic
// one-sub-timestep kernel, templated on the value type and the scheme operator.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ops.cuh"
#include "swept_geom.cuh"
#include "swept_phases.cuh"

namespace swept {

// shared-memory values a swept block needs: two tier rows of C components over
// the M-point window (Section "First-order": the 2 x (n + 2) matrix), plus, for
// Euler, per-tier primitive and face-flux scratch.
template <class Op>
__host__ __device__ inline int64_t swept_smem_values(int M) {
  int64_t v = 2LL * Op::C * M;
  if (Op::C == 3) v += 3LL * M + 3LL * (M + 1) + 3;
  return v;
}

// ---------------------------------------------------------------------------
// one tier of a scalar scheme (heat, KS) on [lo, hi) of the window
// ---------------------------------------------------------------------------
template <typename T, class Op, int STAGE>
__device__ __forceinline__ void scalar_level(T* sm, int M, int out_row, int lo, int hi, int wall,
                                             const typename Op::K& k) {
  constexpr int R = Op::R;
  const T* in = sm + (out_row ^ 1) * M;
  T* out = sm + out_row * M;
  if (wall == NO_WALL) {
    for (int j = lo + (int)threadIdx.x; j < hi; j += (int)blockDim.x) {
      T v[2 * R + 1];
#pragma unroll
      for (int d = 0; d <= 2 * R; ++d) v[d] = in[j + d - R];
      const T p2 = STAGE == 1 ? out[j] : T(0);
      out[j] = Op::template point<STAGE>(v, p2, k);
    }
  } else {
    for (int j = lo + (int)threadIdx.x; j < hi; j += (int)blockDim.x) {
      T v[2 * R + 1];
#pragma unroll
      for (int d = 0; d <= 2 * R; ++d) v[d] = in[nbr(j, d - R, wall)];
      const T p2 = STAGE == 1 ? out[j] : T(0);
      out[j] = Op::template point<STAGE>(v, p2, k);
    }
  }
}

// ---------------------------------------------------------------------------
// one tier of Euler: primitives on [lo-2, hi+2), face fluxes on faces
// [lo, hi] (face f between cells f-1 and f), then the cell update on [lo, hi).
// At a wall face two fluxes exist: the one seen from the right (stored in
// F[f], used by cell f) and from the left (stored in Fw, used by cell f-1).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ typename EulerOp<T>::Prim euler_read_prim(const T* pr, const T* pu, const T* pp, int owner,
                                                                     int d, int wall) {
  typename EulerOp<T>::Prim w;
  const int q = nbr(owner, d, wall);
  w.r = pr[q];
  w.u = through_wall(owner, d, wall) ? -pu[q] : pu[q];
  w.p = pp[q];
  return w;
}

template <typename T>
__device__ __forceinline__ void euler_face(const T* pr, const T* pu, const T* pp, int f, int owner, int wall,
                                           const typename EulerOp<T>::K& k, T& F0, T& F1, T& F2) {
  // cells f-2, f-1, f, f+1 relative to the owner cell
  const auto a = euler_read_prim<T>(pr, pu, pp, owner, f - 2 - owner, wall);
  const auto b = euler_read_prim<T>(pr, pu, pp, owner, f - 1 - owner, wall);
  const auto c = euler_read_prim<T>(pr, pu, pp, owner, f - owner, wall);
  const auto d = euler_read_prim<T>(pr, pu, pp, owner, f + 1 - owner, wall);
  EulerOp<T>::flux(a, b, c, d, k, F0, F1, F2);
}

template <typename T, int STAGE>
__device__ __forceinline__ void euler_level(T* sm, int M, int out_row, int lo, int hi, int wall,
                                            const typename EulerOp<T>::K& k) {
  const T* in0 = sm + ((out_row ^ 1) * 3 + 0) * M;
  const T* in1 = sm + ((out_row ^ 1) * 3 + 1) * M;
  const T* in2 = sm + ((out_row ^ 1) * 3 + 2) * M;
  T* out0 = sm + (out_row * 3 + 0) * M;
  T* out1 = sm + (out_row * 3 + 1) * M;
  T* out2 = sm + (out_row * 3 + 2) * M;
  T* pr = sm + 6 * M;
  T* pu = pr + M;
  T* pp = pu + M;
  T* F0 = pp + M;
  T* F1 = F0 + (M + 1);
  T* F2 = F1 + (M + 1);
  T* Fw = F2 + (M + 1);
  for (int q = lo - 2 + (int)threadIdx.x; q < hi + 2; q += (int)blockDim.x) {
    const auto w = EulerOp<T>::prim(in0[q], in1[q], in2[q], k);
    pr[q] = w.r;
    pu[q] = w.u;
    pp[q] = w.p;
  }
  __syncthreads();
  for (int f = lo + (int)threadIdx.x; f <= hi; f += (int)blockDim.x) {
    if (f == wall) {
      euler_face<T>(pr, pu, pp, f, f, wall, k, F0[f], F1[f], F2[f]);
      euler_face<T>(pr, pu, pp, f, f - 1, wall, k, Fw[0], Fw[1], Fw[2]);
    } else {
      const int owner = (wall == NO_WALL || f > wall) ? f : f - 1;
      euler_face<T>(pr, pu, pp, f, owner, wall, k, F0[f], F1[f], F2[f]);
    }
  }
  __syncthreads();
  for (int j = lo + (int)threadIdx.x; j < hi; j += (int)blockDim.x) {
    const bool wl = (j + 1 == wall);
    const T fp0 = wl ? Fw[0] : F0[j + 1];
    const T fp1 = wl ? Fw[1] : F1[j + 1];
    const T fp2 = wl ? Fw[2] : F2[j + 1];
    const T p20 = STAGE == 1 ? out0[j] : T(0);
    const T p21 = STAGE == 1 ? out1[j] : T(0);
    const T p22 = STAGE == 1 ? out2[j] : T(0);
    out0[j] = EulerOp<T>::template update<STAGE>(fp0, F0[j], in0[j], p20, k);
    out1[j] = EulerOp<T>::template update<STAGE>(fp1, F1[j], in1[j], p21, k);
    out2[j] = EulerOp<T>::template update<STAGE>(fp2, F2[j], in2[j], p22, k);
  }
}

template <typename T, class Op>
struct LevelImpl {
  __device__ __forceinline__ static void run(T* sm, int M, int stage, int out_row, int lo, int hi, int wall,
                                             const typename Op::K& k) {
    if (stage == 0)
      scalar_level<T, Op, 0>(sm, M, out_row, lo, hi, wall, k);
    else
      scalar_level<T, Op, 1>(sm, M, out_row, lo, hi, wall, k);
  }
};
template <typename T>
struct LevelImpl<T, EulerOp<T>> {
  __device__ __forceinline__ static void run(T* sm, int M, int stage, int out_row, int lo, int hi, int wall,
                                             const typename EulerOp<T>::K& k) {
    if (stage == 0)
      euler_level<T, 0>(sm, M, out_row, lo, hi, wall, k);
    else
      euler_level<T, 1>(sm, M, out_row, lo, hi, wall, k);
  }
};

// ---------------------------------------------------------------------------
// device execution context for the pass phases (swept_phases.cuh)
// ---------------------------------------------------------------------------
// Tape: every value a pass computes at absolute tier L is also stored at
// tape[(L - tier0) * C * N + c * N + x] when 0 <= L - tier0 < ntiers (used to
// record the forward tiers the adjoint reads).  `base` is the absolute tier
// of the launch's local tier 0.
template <typename T>
struct Tape {
  T* p = nullptr;
  int64_t tier0 = 0;
  int64_t ntiers = 0;
  int64_t base = 0;
};

template <typename T, class Op, bool TAPE = false>
struct DevCtx {
  T* sm;
  Geom g;
  typename Op::K k;
  const T* u_in;  // may alias u_out (the up-trapezoid reads and writes u)
  T* u_out;
  const T* __restrict__ e_in;
  T* __restrict__ e_out;
  Tape<T> tape;

  template <class F>
  __device__ __forceinline__ void for_range(int lo, int hi, F&& f) {
    for (int i = lo + (int)threadIdx.x; i < hi; i += (int)blockDim.x) f(i);
  }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ T* row(int r, int c) { return sm + (r * Op::C + c) * g.M; }
  __device__ __forceinline__ void load_u(int r, int c, int j, int64_t x) {
    row(r, c)[j] = u_in[c * g.N + wrap_n(x, g.N)];
  }
  __device__ __forceinline__ void store_u(int r, int c, int j, int64_t x) {
    u_out[c * g.N + wrap_n(x, g.N)] = row(r, c)[j];
  }
  __device__ __forceinline__ void load_edge(int r, int c, int j, int64_t e) { row(r, c)[j] = e_in[e]; }
  __device__ __forceinline__ void store_edge(int r, int c, int j, int64_t e) { e_out[e] = row(r, c)[j]; }
  __device__ __forceinline__ void level(int s, int base, int lo, int hi, int64_t origin, int wall) {
    LevelImpl<T, Op>::run(sm, g.M, stage_of(g, s), s & 1, lo, hi, wall, k);
    if (TAPE) {
      // each thread stores the values it computed itself, so no barrier is needed first
      const int64_t slot = tape.base + base + s - tape.tier0;
      if (slot >= 0 && slot < tape.ntiers)
        for (int j = lo + (int)threadIdx.x; j < hi; j += (int)blockDim.x) {
          const int64_t x = wrap_n(origin + j, g.N);
#pragma unroll
          for (int c = 0; c < Op::C; ++c) tape.p[(slot * Op::C + c) * g.N + x] = row(s & 1, c)[j];
        }
    }
    __syncthreads();
  }
};

template <typename T, class Op>
__global__ void __launch_bounds__(1024) k_swept_up(Geom g, typename Op::K k, const T* u_in, T* u_out, T* e_out,
                                                   int hh, int write_top) {
  extern __shared__ __align__(16) unsigned char smraw[];
  DevCtx<T, Op> cx{reinterpret_cast<T*>(smraw), g, k, u_in, u_out, nullptr, e_out, Tape<T>{}};
  run_up(cx, g, (int64_t)blockIdx.x, hh, write_top != 0);
}

template <typename T, class Op>
__global__ void __launch_bounds__(1024) k_swept_diamond(Geom g, typename Op::K k, T* u_out, const T* e_in, T* e_out,
                                                        int odd, int mode, int hh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  DevCtx<T, Op> cx{reinterpret_cast<T*>(smraw), g, k, nullptr, u_out, e_in, e_out, Tape<T>{}};
  run_diamond(cx, g, (int64_t)blockIdx.x, odd, mode, hh);
}

// forward passes that also record every computed tier into a tape
template <typename T, class Op>
__global__ void __launch_bounds__(1024) k_swept_up_tape(Geom g, typename Op::K k, const T* u_in, T* u_out, T* e_out,
                                                        int hh, int write_top, Tape<T> tape) {
  extern __shared__ __align__(16) unsigned char smraw[];
  DevCtx<T, Op, true> cx{reinterpret_cast<T*>(smraw), g, k, u_in, u_out, nullptr, e_out, tape};
  run_up(cx, g, (int64_t)blockIdx.x, hh, write_top != 0);
}

template <typename T, class Op>
__global__ void __launch_bounds__(1024) k_swept_diamond_tape(Geom g, typename Op::K k, T* u_out, const T* e_in,
                                                             T* e_out, int odd, int mode, int hh, Tape<T> tape) {
  extern __shared__ __align__(16) unsigned char smraw[];
  DevCtx<T, Op, true> cx{reinterpret_cast<T*>(smraw), g, k, nullptr, u_out, e_in, e_out, tape};
  run_diamond(cx, g, (int64_t)blockIdx.x, odd, mode, hh);
}

// ---------------------------------------------------------------------------
// adjoint passes: the same swept schedule on lam, reverse tier L reading the
// forward state of tape slot (S K - L) at the same point, and accumulating the
// parameter derivative per thread; each block adds its sum to slot[block]
// (blocks of later launches add to the same slot in launch order, so the
// result is deterministic).
// ---------------------------------------------------------------------------
template <typename T, class AOp>
__device__ __forceinline__ void adjoint_level(T* sm, int M, int stage, int out_row, int lo, int hi, int wall,
                                              int64_t origin, int64_t N, const T* fwd, const typename AOp::K& k,
                                              KahanAcc& acc) {
  constexpr int R = AOp::R;
  const T* in = sm + (out_row ^ 1) * M;
  T* out = sm + out_row * M;
  for (int j = lo + (int)threadIdx.x; j < hi; j += (int)blockDim.x) {
    T v[2 * R + 1];
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) v[d] = in[nbr(j, d - R, wall)];
    const T w = fwd[wrap_n(origin + j, N)];
    if (stage == 0)
      out[j] = AOp::template point<0>(v, T(0), w, k, acc);
    else
      out[j] = AOp::template point<1>(v, out[j], w, k, acc);
  }
}

template <typename T, class AOp>
struct AdjCtx {
  T* sm;
  Geom g;
  typename AOp::K k;
  const T* u_in;
  T* u_out;
  const T* __restrict__ e_in;
  T* __restrict__ e_out;
  const T* __restrict__ tape;  // forward tiers 0 .. S K of the segment, N values each
  int64_t top;                 // S K: reverse tier L reads forward slot top - L
  int64_t base;                // absolute reverse tier of the launch's local tier 0
  KahanAcc acc;

  template <class F>
  __device__ __forceinline__ void for_range(int lo, int hi, F&& f) {
    for (int i = lo + (int)threadIdx.x; i < hi; i += (int)blockDim.x) f(i);
  }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ T* row(int r, int c) { return sm + (r * AOp::C + c) * g.M; }
  __device__ __forceinline__ void load_u(int r, int c, int j, int64_t x) {
    row(r, c)[j] = u_in[c * g.N + wrap_n(x, g.N)];
  }
  __device__ __forceinline__ void store_u(int r, int c, int j, int64_t x) {
    u_out[c * g.N + wrap_n(x, g.N)] = row(r, c)[j];
  }
  __device__ __forceinline__ void load_edge(int r, int c, int j, int64_t e) { row(r, c)[j] = e_in[e]; }
  __device__ __forceinline__ void store_edge(int r, int c, int j, int64_t e) { e_out[e] = row(r, c)[j]; }
  __device__ __forceinline__ void level(int s, int b, int lo, int hi, int64_t origin, int wall) {
    const int64_t L = base + b + s;
    adjoint_level<T, AOp>(sm, g.M, stage_of(g, s), s & 1, lo, hi, wall, origin, g.N, tape + (top - L) * g.N, k,
                          acc);
    __syncthreads();
  }
};

// double-double arithmetic for the parameter-derivative reduction
struct DD {
  double hi, lo;
};
__device__ __forceinline__ DD two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bp = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bp)), __dsub_rn(b, bp));
  return DD{s, e};
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  const DD s = two_sum(a.hi, b.hi);
  return two_sum(s.hi, __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo)));
}

// deterministic block sum of one double-double per thread (blockDim.x a
// multiple of 32); the result is valid in thread 0
__device__ __forceinline__ DD block_sum(DD v, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) {
    DD w;
    w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, w);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    scratch[2 * warp] = v.hi;
    scratch[2 * warp + 1] = v.lo;
  }
  __syncthreads();
  DD t{0.0, 0.0};
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = dd_add(t, DD{scratch[2 * w], scratch[2 * w + 1]});
  return t;
}

// slots hold one double-double (hi, lo) per block
__device__ __forceinline__ void add_to_slot(double* slots, DD t) {
  const DD r = dd_add(DD{slots[2 * blockIdx.x], slots[2 * blockIdx.x + 1]}, t);
  slots[2 * blockIdx.x] = r.hi;
  slots[2 * blockIdx.x + 1] = r.lo;
}

template <typename T, class AOp>
__global__ void __launch_bounds__(1024) k_adj_up(Geom g, typename AOp::K k, const T* u_in, T* u_out, T* e_out, int hh,
                                                 int write_top, const T* tape, int64_t top, int64_t base,
                                                 double* slots) {
  extern __shared__ __align__(16) unsigned char smraw[];
  AdjCtx<T, AOp> cx{reinterpret_cast<T*>(smraw), g, k, u_in, u_out, nullptr, e_out, tape, top, base, KahanAcc{}};
  run_up(cx, g, (int64_t)blockIdx.x, hh, write_top != 0);
  const DD t = block_sum(DD{cx.acc.s, -cx.acc.c}, reinterpret_cast<double*>(smraw));
  if (threadIdx.x == 0) add_to_slot(slots, t);
}

template <typename T, class AOp>
__global__ void __launch_bounds__(1024) k_adj_diamond(Geom g, typename AOp::K k, T* u_out, const T* e_in, T* e_out,
                                                      int odd, int mode, int hh, const T* tape, int64_t top,
                                                      int64_t base, double* slots) {
  extern __shared__ __align__(16) unsigned char smraw[];
  AdjCtx<T, AOp> cx{reinterpret_cast<T*>(smraw), g, k, nullptr, u_out, e_in, e_out, tape, top, base, KahanAcc{}};
  run_diamond(cx, g, (int64_t)blockIdx.x, odd, mode, hh);
  const DD t = block_sum(DD{cx.acc.s, -cx.acc.c}, reinterpret_cast<double*>(smraw));
  if (threadIdx.x == 0) add_to_slot(slots, t);
}

// out[0] = double-double sum of the n (hi, lo) slots in index order (one thread: deterministic)
static __global__ void k_sum_slots(const double* slots, int64_t n, double* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DD t{0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) t = dd_add(t, DD{slots[2 * i], slots[2 * i + 1]});
    out[0] = __dadd_rn(t.hi, t.lo);
  }
}

// ---------------------------------------------------------------------------
// classic decomposition: one sub-timestep per launch through global memory
// (Section "Classic scheme", Fig. ClassicCode)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t classic_nbr(int64_t i, int64_t N, int bc, bool* flip) {
  *flip = false;
  if (i >= 0 && i < N) return i;
  if (bc == 0) return i < 0 ? i + N : i - N;
  *flip = true;
  return i < 0 ? -1 - i : 2 * N - 1 - i;
}

template <typename T, class Op, int STAGE>
__global__ void __launch_bounds__(256) k_classic(int64_t N, int bc, typename Op::K k, const T* __restrict__ in,
                                                 T* out) {
  constexpr int R = Op::R;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  T v[2 * R + 1];
  if (i >= R && i < N - R) {
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) v[d] = in[i + d - R];
  } else {
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) {
      bool f;
      v[d] = in[classic_nbr(i + d - R, N, bc, &f)];
    }
  }
  const T p2 = STAGE == 1 ? out[i] : T(0);
  out[i] = Op::template point<STAGE>(v, p2, k);
}

// Euler classic stage: a block of blockDim.x cells stages conserved values and
// primitives of its cells plus 2 halo cells per side in shared memory, computes
// its blockDim.x + 1 face fluxes once, then updates its cells.
template <typename T, int STAGE>
__global__ void __launch_bounds__(256) k_classic_euler(int64_t N, int bc, typename EulerOp<T>::K k,
                                                       const T* __restrict__ in, T* out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int B = blockDim.x;
  const int Wn = B + 4;
  T* pr = reinterpret_cast<T*>(smraw);
  T* pu = pr + Wn;
  T* pp = pu + Wn;
  T* F0 = pp + Wn;
  T* F1 = F0 + (B + 1);
  T* F2 = F1 + (B + 1);
  const int64_t i0 = (int64_t)blockIdx.x * B;
  for (int t = threadIdx.x; t < Wn; t += B) {
    const int64_t x = i0 - 2 + t;
    if (x - 2 >= N) continue;  // beyond the last block's last face stencil
    bool flip;
    const int64_t c = classic_nbr(x, N, bc, &flip);
    const T m = flip ? -in[N + c] : in[N + c];
    const auto w = EulerOp<T>::prim(in[c], m, in[2 * N + c], k);
    pr[t] = w.r;
    pu[t] = w.u;
    pp[t] = w.p;
  }
  __syncthreads();
  for (int f = threadIdx.x; f <= B; f += B) {
    if (i0 + f > N) continue;
    typename EulerOp<T>::Prim a{pr[f], pu[f], pp[f]}, b{pr[f + 1], pu[f + 1], pp[f + 1]},
        c{pr[f + 2], pu[f + 2], pp[f + 2]}, d{pr[f + 3], pu[f + 3], pp[f + 3]};
    EulerOp<T>::flux(a, b, c, d, k, F0[f], F1[f], F2[f]);
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t i = i0 + t;
  if (i >= N) return;
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    const T* F = cc == 0 ? F0 : (cc == 1 ? F1 : F2);
    const T p2 = STAGE == 1 ? out[cc * N + i] : T(0);
    out[cc * N + i] = EulerOp<T>::template update<STAGE>(F[t + 1], F[t], in[cc * N + i], p2, k);
  }
}

template <typename T>
__global__ void k_copy(int64_t n, const T* __restrict__ src, T* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace swept
