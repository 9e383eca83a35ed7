// CUDA kernels: swept passes (up-triangle, diamond, down/gap) and the classic
// one-sub-timestep kernel, templated on the value type and the scheme operator.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "debug_check.cuh"
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

// Strided mapping with two points per thread per trip (j and j + blockDim.x):
// both windows are loaded before either result is stored, so each thread has
// two independent update chains in flight.
template <typename T, class Op, int STAGE>
__device__ __forceinline__ void strided2_level(T* sm, int M, int out_row, int lo, int hi, const typename Op::K& k) {
  constexpr int R = Op::R;
  const T* in = sm + (out_row ^ 1) * M;
  T* out = sm + out_row * M;
  const int T2 = 2 * (int)blockDim.x;
  const int lim = hi + R - 1;
  for (int j = lo + (int)threadIdx.x; j < hi; j += T2) {
    const int j2 = j + (int)blockDim.x;
    T va[2 * R + 1], vb[2 * R + 1];
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) {
      va[d] = in[j + d - R];
      vb[d] = in[min(j2 + d - R, lim)];
    }
    const T pa = STAGE == 1 ? out[j] : T(0);
    const T pb = STAGE == 1 ? out[min(j2, hi - 1)] : T(0);
    const T ra = Op::template point<STAGE>(va, pa, k);
    const T rb = Op::template point<STAGE>(vb, pb, k);
    out[j] = ra;
    if (j2 < hi) out[j2] = rb;
  }
}

// Radius-2 tier with each thread advancing the aligned pair (j, j + 1), j
// even: its six inputs j-2 .. j+3 come from three paired loads (float2) and
// both results go out in one paired store, 2.25 shared-memory instructions a
// point instead of 6.5.  Needs even lo and hi and an even row
// stride (every KS tier of a tile whose width is a multiple of 8 has even
// bounds).  Each point is the same Op::point on the same operands.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

template <typename T, class Op, int STAGE>
__device__ __forceinline__ void paired_level(T* sm, int M, int out_row, int lo, int hi, const typename Op::K& k) {
  static_assert(Op::R == 2, "paired tiers are for radius-2 stencils");
  using T2 = typename Pair<T>::type;
  const T2* in = reinterpret_cast<const T2*>(sm + (out_row ^ 1) * M);
  T2* out = reinterpret_cast<T2*>(sm + out_row * M);
  for (int jp = (lo >> 1) + (int)threadIdx.x; jp < (hi >> 1); jp += (int)blockDim.x) {
    const T2 a = in[jp - 1], b = in[jp], c = in[jp + 1];
    const T v[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
    const T2 p2 = STAGE == 1 ? out[jp] : T2{T(0), T(0)};
    T2 r;
    r.x = Op::template point<STAGE>(&v[0], p2.x, k);
    r.y = Op::template point<STAGE>(&v[1], p2.y, k);
    out[jp] = r;
  }
}

template <typename T, class Op, int STAGE>
__device__ __forceinline__ void scalar_level_any(T* sm, int M, int out_row, int lo, int hi, int wall, int chunk,
                                                 const typename Op::K& k) {
  // FP32 only: in FP64 a warp instruction holds the FP64 pipe for 64 cycles
  // whatever its active lanes, and pairs double the partial-warp waste at the
  // triangle tips (measured 4 % slower on the FP64 KS workload)
  if constexpr (Op::R == 2 && sizeof(T) == 4) {
    if (wall == NO_WALL && chunk <= 1 && ((lo | hi | M) & 1) == 0) {
      paired_level<T, Op, STAGE>(sm, M, out_row, lo, hi, k);
      return;
    }
  }
  if (wall != NO_WALL || chunk <= 1) {
    scalar_level<T, Op, STAGE>(sm, M, out_row, lo, hi, wall, k);
    return;
  }
  strided2_level<T, Op, STAGE>(sm, M, out_row, lo, hi, k);
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

// One side of face f for the two-threads-per-face flux phase, with one code
// path for both sides (no divergence within a lane pair): side 0 (left)
// reconstructs p1 + h from cells f-2, f-1, f; side 1 (right) p1 - h from
// cells f-1, f, f+1, where h = 1/2 minmod(p1 - p0, p2 - p1).  Adding -h is
// the same IEEE operation as subtracting h, so both sides equal
// EulerOp::left_side / right_side bit for bit.
template <typename T>
__device__ __forceinline__ typename EulerOp<T>::Side euler_side(const T* pr, const T* pu, const T* pp, int f,
                                                                int owner, int wall, int side,
                                                                const typename EulerOp<T>::K& k) {
  const auto p0 = euler_read_prim<T>(pr, pu, pp, owner, f - 2 + side - owner, wall);
  const auto p1 = euler_read_prim<T>(pr, pu, pp, owner, f - 1 + side - owner, wall);
  const auto p2 = euler_read_prim<T>(pr, pu, pp, owner, f + side - owner, wall);
  typename EulerOp<T>::Side X;
  const T hr = mul_rn(T(0.5), minmod(sub_rn(p1.r, p0.r), sub_rn(p2.r, p1.r)));
  const T hu = mul_rn(T(0.5), minmod(sub_rn(p1.u, p0.u), sub_rn(p2.u, p1.u)));
  const T hp = mul_rn(T(0.5), minmod(sub_rn(p1.p, p0.p), sub_rn(p2.p, p1.p)));
  X.r = add_rn(p1.r, side ? -hr : hr);
  X.u = add_rn(p1.u, side ? -hu : hu);
  X.p = add_rn(p1.p, side ? -hp : hp);
  EulerOp<T>::finish_side(X, k);
  return X;
}

// the flux of face f by a lane pair (lanes 2t, 2t+1 of `mask`): each lane
// builds its side, the pair swaps sides by shuffle, the left lane forms
// F0, F1 and the right lane F2; stored only when `store`
template <typename T>
__device__ __forceinline__ void euler_face_pair(const T* pr, const T* pu, const T* pp, int f, int owner, int wall,
                                                int side, bool store, unsigned mask,
                                                const typename EulerOp<T>::K& k, T* F0, T* F1, T* F2) {
  using Side = typename EulerOp<T>::Side;
  const Side X = euler_side<T>(pr, pu, pp, f, owner, wall, side, k);
  Side Y;
  Y.r = __shfl_xor_sync(mask, X.r, 1);
  Y.u = __shfl_xor_sync(mask, X.u, 1);
  Y.p = __shfl_xor_sync(mask, X.p, 1);
  Y.m = __shfl_xor_sync(mask, X.m, 1);
  Y.E = __shfl_xor_sync(mask, X.E, 1);
  Y.sp = __shfl_xor_sync(mask, X.sp, 1);
  const Side L = side ? Y : X;
  const Side R = side ? X : Y;
  const T s = EulerOp<T>::smax(L, R);
  if (side == 0) {
    const T a0 = EulerOp<T>::flux0(L, R, s);
    const T a1 = EulerOp<T>::flux1(L, R, s);
    if (store) {
      *F0 = a0;
      *F1 = a1;
    }
  } else {
    const T a2 = EulerOp<T>::flux2(L, R, s);
    if (store) *F2 = a2;
  }
}

template <typename T, int STAGE, bool PAIR = false>
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
  // Work items of the flux phase: faces lo..hi (item f - lo), and for a wall
  // face inside the range also its flux seen from the left cell (item nf),
  // handed to its own thread so the wall costs no thread a second flux.
  const int nf = hi - lo + 1;
  const int nitems = nf + ((wall != NO_WALL && wall >= lo && wall <= hi) ? 1 : 0);
  if (!PAIR && wall == NO_WALL) {
    // no wall in the window: faces read their four cells directly
    for (int f = lo + (int)threadIdx.x; f <= hi; f += (int)blockDim.x) {
      const typename EulerOp<T>::Prim a{pr[f - 2], pu[f - 2], pp[f - 2]}, b{pr[f - 1], pu[f - 1], pp[f - 1]},
          c{pr[f], pu[f], pp[f]}, d{pr[f + 1], pu[f + 1], pp[f + 1]};
      EulerOp<T>::flux(a, b, c, d, k, F0[f], F1[f], F2[f]);
    }
  } else if (!PAIR) {
    for (int i = (int)threadIdx.x; i < nitems; i += (int)blockDim.x) {
      if (i < nf) {
        const int f = lo + i;
        const int owner = (wall == NO_WALL || f >= wall) ? f : f - 1;
        euler_face<T>(pr, pu, pp, f, owner, wall, k, F0[f], F1[f], F2[f]);
      } else {
        euler_face<T>(pr, pu, pp, wall, wall - 1, wall, k, Fw[0], Fw[1], Fw[2]);
      }
    }
  } else {
    // two threads per item; the trip count is the same for all lanes of a
    // warp (a warp leaves once its first pair is past the last item), so
    // every lane of a working warp reaches the shuffles (pairs past the end
    // recompute the last item and store nothing)
    const int half = (int)blockDim.x >> 1;
    const int side = (int)threadIdx.x & 1;
    const int t = (int)threadIdx.x >> 1;
    const int t_warp = (int)(threadIdx.x & ~31u) >> 1;  // first pair of this warp
    for (int base = 0; base + t_warp < nitems; base += half) {
      const bool act = base + t < nitems;
      const int i = act ? base + t : nitems - 1;
      const bool second = i == nf;  // the wall face seen from its left cell
      const int f = second ? wall : lo + i;
      const int owner = second ? wall - 1 : ((wall == NO_WALL || f >= wall) ? f : f - 1);
      euler_face_pair<T>(pr, pu, pp, f, owner, wall, side, act, 0xffffffffu, k, second ? Fw : F0 + f,
                         second ? Fw + 1 : F1 + f, second ? Fw + 2 : F2 + f);
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
                                             int chunk, const typename Op::K& k) {
    if (stage == 0)
      scalar_level_any<T, Op, 0>(sm, M, out_row, lo, hi, wall, chunk, k);
    else
      scalar_level_any<T, Op, 1>(sm, M, out_row, lo, hi, wall, chunk, k);
  }
};
// Euler: chunk 2 = two threads per face in the flux phase
template <typename T>
struct LevelImpl<T, EulerOp<T>> {
  __device__ __forceinline__ static void run(T* sm, int M, int stage, int out_row, int lo, int hi, int wall,
                                             int chunk, const typename EulerOp<T>::K& k) {
    if (chunk == 2) {
      if (stage == 0)
        euler_level<T, 0, true>(sm, M, out_row, lo, hi, wall, k);
      else
        euler_level<T, 1, true>(sm, M, out_row, lo, hi, wall, k);
    } else {
      if (stage == 0)
        euler_level<T, 0>(sm, M, out_row, lo, hi, wall, k);
      else
        euler_level<T, 1>(sm, M, out_row, lo, hi, wall, k);
    }
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
  using value_type = T;
  using op_type = Op;
  static constexpr int kR = Op::R, kC = Op::C;
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
    if (dbg::win(g.M, r, c, kC, j)) row(r, c)[j] = u_in[c * g.N + wrap_n(x, g.N)];
  }
  __device__ __forceinline__ void store_u(int r, int c, int j, int64_t x) {
    if (dbg::win(g.M, r, c, kC, j)) u_out[c * g.N + wrap_n(x, g.N)] = row(r, c)[j];
  }
  __device__ __forceinline__ void load_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(g.M, r, c, kC, j) && dbg::in_range(e, edge_slots(g) * g.E, dbg::EDGE)) row(r, c)[j] = e_in[e];
  }
  __device__ __forceinline__ void store_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(g.M, r, c, kC, j) && dbg::in_range(e, edge_slots(g) * g.E, dbg::EDGE)) e_out[e] = row(r, c)[j];
  }
  __device__ __forceinline__ void level(int s, int base, int lo, int hi, int64_t origin, int wall) {
    if (dbg::level(g.M, lo, hi, kR)) LevelImpl<T, Op>::run(sm, g.M, stage_c<Op>(s), s & 1, lo, hi, wall, g.chunk, k);
    if (TAPE) {
      // the tier's mapping of points to threads (strided or paired)
      // need not match this loop's, so the tier must be complete first
      __syncthreads();
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


// ---------------------------------------------------------------------------
// Tiers in registers (scalar schemes, Geom::P > 0): the block is one warp and
// owns one tile of W = 32 P points.  Lane l keeps window points R + l P + i
// (i < P) of both tier rows in registers; the halo points [0, R) and
// [W + R, W + 2R), which only ever hold inserted edges, are kept by every lane
// and used by lanes 0 and 31.  A tier takes the R points beyond each end of a
// lane's run from the neighbouring lanes with __shfl_up_sync/__shfl_down_sync,
// so it costs no shared-memory access and no barrier.  The loads and stores
// of a pass (tile, edges) still go through the shared-memory rows of the base
// context: the rows move into registers at the first tier of a pass and back
// (then __syncwarp) before the first load/store loop after the tiers.  Every
// tier evaluates the same Op::point on the same operands in the same order as
// the shared-memory tiers, so the two give identical results.
// ---------------------------------------------------------------------------
template <class Base, int P>
struct RegCtx : Base {
  using T = typename Base::value_type;
  using Op = typename Base::op_type;
  static constexpr int R = Op::R;
  static_assert(Op::C == 1 && P >= 1, "register tiers need a scalar scheme");
  T a[P], b[P];            // rows 0 (even tiers) and 1 (odd tiers)
  T ha[2 * R], hb[2 * R];  // halo of rows 0 / 1: [0, R) -> points 0..R-1, [R, 2R) -> points W+R..W+2R-1
  bool in_regs;

  __device__ __forceinline__ explicit RegCtx(const Base& base) : Base(base), in_regs(false) {}

  __device__ __forceinline__ static int lane() { return (int)(threadIdx.x & 31u); }
  __device__ __forceinline__ void fill() {
    const T* r0 = this->row(0, 0);
    const T* r1 = this->row(1, 0);
    const int p0 = R + lane() * P;
#pragma unroll
    for (int i = 0; i < P; ++i) {
      a[i] = r0[p0 + i];
      b[i] = r1[p0 + i];
    }
    const int W = this->g.W;
#pragma unroll
    for (int d = 0; d < R; ++d) {
      ha[d] = r0[d];
      hb[d] = r1[d];
      ha[R + d] = r0[W + R + d];
      hb[R + d] = r1[W + R + d];
    }
    in_regs = true;
  }
  __device__ __forceinline__ void spill() {
    T* r0 = this->row(0, 0);
    T* r1 = this->row(1, 0);
    const int p0 = R + lane() * P;
#pragma unroll
    for (int i = 0; i < P; ++i) {
      r0[p0 + i] = a[i];
      r1[p0 + i] = b[i];
    }
    __syncwarp();
    in_regs = false;
  }
  template <class F>
  __device__ __forceinline__ void for_range(int lo, int hi, F&& f) {
    if (in_regs) spill();
    Base::for_range(lo, hi, f);
  }
  // tier s on [lo, hi): into row s&1 from row (s-1)&1; stage (s-1) mod S
  __device__ __forceinline__ void level(int s, int, int lo, int hi, int64_t, int wall) {
    if (!dbg::level(this->g.M, lo, hi, R)) return;
    if (!in_regs) fill();
    if (s & 1)
      tier<0>(a, ha, b, lo, hi, wall);
    else
      tier<Op::S == 1 ? 0 : 1>(b, hb, a, lo, hi, wall);
  }
  template <int STAGE>
  __device__ __forceinline__ void tier(const T (&src)[P], const T (&hs)[2 * R], T (&dst)[P], int lo, int hi,
                                       int wall) {
    const int ln = lane();
    T w[P + 2 * R];  // points p0 - R .. p0 + P + R - 1 of the source tier
#pragma unroll
    for (int d = 0; d < R; ++d) {
      // left halo point d is window point ln P + d: element el of lane ln - kl, or, for the
      // first kl lanes, the window's own halo hs[ln P + d] (kl = 1 when P >= R)
      const int kl = (R - d + P - 1) / P, el = d - R + kl * P;
      const T x = __shfl_up_sync(0xffffffffu, src[el], kl);
      T hx = hs[d];
#pragma unroll
      for (int m = 1; m < kl; ++m)
        if (ln == m) hx = hs[m * P + d];
      w[d] = ln < kl ? hx : x;
      // right halo point d is window point R + (ln + 1) P + d: element er of lane ln + kr, or,
      // for the last kr lanes, hs[R + d - m P] on lane 31 - m (kr = 1 when P >= R)
      const int kr = 1 + d / P, er = d - (kr - 1) * P;
      const T y = __shfl_down_sync(0xffffffffu, src[er], kr);
      T hy = hs[R + d];
#pragma unroll
      for (int m = 1; m < kr; ++m)
        if (ln == 31 - m) hy = hs[R + d - m * P];
      w[R + P + d] = ln > 31 - kr ? hy : y;
    }
#pragma unroll
    for (int i = 0; i < P; ++i) w[R + i] = src[i];
    const int p0 = R + ln * P;
    if (wall == NO_WALL) {
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const T r = Op::template point<STAGE>(&w[i], dst[i], this->k);
        if (p0 + i >= lo && p0 + i < hi) dst[i] = r;
      }
    } else {
      // across a mirror wall the neighbour read is the mirror image, which
      // lies within R of the point on its own side (nbr), i.e. inside w
#pragma unroll
      for (int i = 0; i < P; ++i) {
        T v[2 * R + 1];
#pragma unroll
        for (int d = 0; d <= 2 * R; ++d) {
          const int q = nbr(p0 + i, d - R, wall) - (p0 + i);
          T x = w[i + R];
#pragma unroll
          for (int e = 0; e <= 2 * R; ++e)
            if (q == e - R) x = w[i + e];
          v[d] = x;
        }
        const T r = Op::template point<STAGE>(v, dst[i], this->k);
        if (p0 + i >= lo && p0 + i < hi) dst[i] = r;
      }
    }
  }
};

// the context of a pass: Base itself (P = 0) or Base with its tiers in registers.
// The register-tier kernels run one warp per block and are compiled for 16
// co-resident blocks per SM (at most 128 registers per thread).
template <class Base, int P>
struct WithTiers {
  using type = RegCtx<Base, P>;
};
template <class Base>
struct WithTiers<Base, 0> {
  using type = Base;
};
template <int P, class Base>
__device__ __forceinline__ typename WithTiers<Base, P>::type tiers_ctx(const Base& base) {
  return typename WithTiers<Base, P>::type(base);
}

// Launch bounds of the swept kernels.  P > 0: one warp per block, 16 blocks
// per SM.  Shared-memory tiers: MAXT threads at most; MAXT = 1024 caps a
// thread at 64 registers; MAXT = 256 (the variant blocks of up to 256 threads
// run) at 85 with 3 blocks per SM, which measured faster on the Euler
// workloads than 2 blocks of up to 128 registers.
#define SWEPT_BOUNDS(P, MAXT) __launch_bounds__((P) > 0 ? 32 : (MAXT), (P) > 0 ? 16 : ((MAXT) <= 256 ? 3 : 1))

// ---------------------------------------------------------------------------
// persistent single-problem swept kernel: the launch sequence of
// for_each_launch as one queue of (pass k, tile b) items, item = k * nt + b,
// claimed in order by a grid no larger than the co-resident blocks.  Before a
// pass-k item a block waits (bounded) until the tiles it reads have finished
// pass k-1 (the zig-zag dependencies; they also cover reuse of the ping-pong
// edge buffers), runs the pass phases, and publishes done[b] = k.  Global
// reads go through L2 (ld.global.cg): other SMs write these buffers while the
// block runs.
// ---------------------------------------------------------------------------
struct PersistCtl {
  int* done;                  // nt tile counters, -1 before pass 0
  unsigned long long* queue;  // next item
  int* error;                 // SWEPT_ETIMEOUT (4) once a wait ran out
  uint32_t spin_limit;
  int64_t start_item;         // the first item claimed (0; > 0 only to exercise the timeout path)
};

template <typename T, class Op>
struct PDevCtx {
  using value_type = T;
  using op_type = Op;
  static constexpr int kR = Op::R, kC = Op::C;
  T* sm;
  Geom g;
  typename Op::K k;
  T* u;
  const T* e_in;
  T* e_out;

  template <class F>
  __device__ __forceinline__ void for_range(int lo, int hi, F&& f) {
    for (int i = lo + (int)threadIdx.x; i < hi; i += (int)blockDim.x) f(i);
  }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ T* row(int r, int c) { return sm + (r * Op::C + c) * g.M; }
  __device__ __forceinline__ void load_u(int r, int c, int j, int64_t x) {
    if (dbg::win(g.M, r, c, kC, j)) row(r, c)[j] = __ldcg(u + c * g.N + wrap_n(x, g.N));
  }
  __device__ __forceinline__ void store_u(int r, int c, int j, int64_t x) {
    if (dbg::win(g.M, r, c, kC, j)) u[c * g.N + wrap_n(x, g.N)] = row(r, c)[j];
  }
  __device__ __forceinline__ void load_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(g.M, r, c, kC, j) && dbg::in_range(e, edge_slots(g) * g.E, dbg::EDGE)) row(r, c)[j] = __ldcg(e_in + e);
  }
  __device__ __forceinline__ void store_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(g.M, r, c, kC, j) && dbg::in_range(e, edge_slots(g) * g.E, dbg::EDGE)) e_out[e] = row(r, c)[j];
  }
  __device__ __forceinline__ void level(int s, int, int lo, int hi, int64_t, int wall) {
    if (dbg::level(g.M, lo, hi, kR)) LevelImpl<T, Op>::run(sm, g.M, stage_c<Op>(s), s & 1, lo, hi, wall, g.chunk, k);
    __syncthreads();
  }
};

// bounded wait for *flag >= need; gives up at the limit or once any block has
// recorded an error
__device__ __forceinline__ bool persist_wait(const int* flag, int need, const PersistCtl& c) {
  for (uint32_t i = 0;; ++i) {
    if (*(volatile const int*)flag >= need) return true;
    if (i >= c.spin_limit || *(volatile const int*)c.error != 0) return false;
    __nanosleep(128);
  }
}

template <typename T, class Op, int P = 0, int MAXT = 1024>
__global__ void SWEPT_BOUNDS(P, MAXT) k_swept_persist(Geom g, typename Op::K k, T* u, T* e0, T* e1, int64_t n_sub,
                                                        PersistCtl ctl) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int64_t s_item;
  __shared__ int s_ok;
  const int q = (int)(n_sub / g.h), rem = (int)(n_sub % g.h);
  const int main_passes = q > 0 ? q + 1 : 0;
  const int64_t total = (int64_t)(main_passes + (rem > 0 ? 2 : 0)) * g.nt;
  T* eb[2] = {e0, e1};
  for (;;) {
    if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(ctl.queue, 1ULL) + ctl.start_item;
    __syncthreads();
    const int64_t item = s_item;
    if (item >= total) break;
    const int kp = (int)(item / g.nt);
    const int64_t b = item - (int64_t)kp * g.nt;
    if (threadIdx.x == 0) {
      bool ok = *(volatile int*)ctl.error == 0;
      int64_t dep_tile[3];
      int dep_need[3];
      const int ndep = persist_deps(g, n_sub, kp, b, dep_tile, dep_need);
      for (int i = 0; ok && i < ndep; ++i)
        ok = dbg::in_range(dep_tile[i], g.nt, dbg::COUNTER) && persist_wait(ctl.done + dep_tile[i], dep_need[i], ctl);
      if (!ok) atomicCAS(ctl.error, 0, 4);
      s_ok = ok;
      __threadfence();
    }
    __syncthreads();
    if (!s_ok) break;
    auto cx = tiers_ctx<P>(PDevCtx<T, Op>{reinterpret_cast<T*>(smraw), g, k, u, nullptr, nullptr});
    if (kp < main_passes) {
      if (kp == 0) {
        cx.e_out = eb[0];
        run_up(cx, g, b, g.h, false);
      } else {
        cx.e_in = eb[(kp - 1) & 1];
        cx.e_out = eb[kp & 1];
        run_diamond(cx, g, b, kp & 1, kp == q ? MODE_DOWN : MODE_DIAMOND, g.h);
      }
    } else if (kp == main_passes) {
      cx.e_out = eb[0];
      run_up(cx, g, b, rem, true);
    } else {
      cx.e_in = eb[0];
      cx.e_out = eb[1];
      run_diamond(cx, g, b, 1, MODE_GAP, rem);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(ctl.done + b, kp);
  }
}

// ---------------------------------------------------------------------------
// cluster-resident swept kernel: the whole grid (nt <= 16 tiles) is one
// thread-block cluster, block b owning tile b for the entire solve.  Edges are
// exported into a ping-pong area of the block's own shared memory and read by
// the neighbour block straight from there through distributed shared memory
// (cluster.map_shared_rank); a cluster barrier separates the passes.  No
// global edge buffers and no per-pass launches.  The state is read at the
// first pass and written by the down-triangle and remainder passes only.
// ---------------------------------------------------------------------------
template <typename T, class Op>
struct ClusterCtx {
  using value_type = T;
  using op_type = Op;
  static constexpr int kR = Op::R, kC = Op::C;
  T* sm;         // the block's window rows (and Euler scratch)
  T* ex_in;      // export area of the previous pass (read remotely)
  T* ex_out;     // export area this pass writes (own tile's edges)
  Geom g;
  typename Op::K k;
  T* u;
  unsigned my_rank;

  template <class F>
  __device__ __forceinline__ void for_range(int lo, int hi, F&& f) {
    for (int i = lo + (int)threadIdx.x; i < hi; i += (int)blockDim.x) f(i);
  }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ T* row(int r, int c) { return sm + (r * Op::C + c) * g.M; }
  __device__ __forceinline__ void load_u(int r, int c, int j, int64_t x) {
    if (dbg::win(g.M, r, c, kC, j)) row(r, c)[j] = __ldcg(u + c * g.N + wrap_n(x, g.N));
  }
  __device__ __forceinline__ void store_u(int r, int c, int j, int64_t x) {
    if (dbg::win(g.M, r, c, kC, j)) u[c * g.N + wrap_n(x, g.N)] = row(r, c)[j];
  }
  __device__ __forceinline__ void load_edge(int r, int c, int j, int64_t e) {
    if (!dbg::win(g.M, r, c, kC, j) || !dbg::in_range(e, edge_slots(g) * g.E, dbg::EDGE)) return;
    const unsigned tile = (unsigned)(e / g.E);
    const T* src = cooperative_groups::this_cluster().map_shared_rank(ex_in + (e - (int64_t)tile * g.E), tile);
    row(r, c)[j] = *src;
  }
  __device__ __forceinline__ void store_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(g.M, r, c, kC, j) && dbg::in_range(e - (int64_t)my_rank * g.E, g.E, dbg::EDGE))
      ex_out[e - (int64_t)my_rank * g.E] = row(r, c)[j];
  }
  __device__ __forceinline__ void level(int s, int, int lo, int hi, int64_t, int wall) {
    if (dbg::level(g.M, lo, hi, kR)) LevelImpl<T, Op>::run(sm, g.M, stage_c<Op>(s), s & 1, lo, hi, wall, g.chunk, k);
    __syncthreads();
  }
};

template <typename T, class Op, int P = 0>
__global__ void __launch_bounds__(P > 0 ? 32 : 1024, P > 0 ? 16 : 1) k_swept_cluster(Geom g, typename Op::K k, T* u, int64_t n_sub,
                                                        int64_t smem_values) {
  extern __shared__ __align__(16) unsigned char smraw[];
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  T* sm = reinterpret_cast<T*>(smraw);
  T* ex[2] = {sm + smem_values, sm + smem_values + g.E};
  const unsigned b = cluster.block_rank();
  auto cx = tiers_ctx<P>(ClusterCtx<T, Op>{sm, ex[1], ex[0], g, k, u, b});
  const int q = (int)(n_sub / g.h), rem = (int)(n_sub % g.h);
  if (q > 0) {
    cx.ex_out = ex[0];
    run_up(cx, g, (int64_t)b, g.h, false);
    cluster.sync();
    for (int p = 1; p <= q; ++p) {
      cx.ex_in = ex[(p - 1) & 1];
      cx.ex_out = ex[p & 1];
      run_diamond(cx, g, (int64_t)b, p & 1, p == q ? MODE_DOWN : MODE_DIAMOND, g.h);
      cluster.sync();  // edges of pass p complete (and, after the down pass, the state)
    }
  }
  if (rem > 0) {
    cx.ex_out = ex[0];
    run_up(cx, g, (int64_t)b, rem, true);
    cluster.sync();
    cx.ex_in = ex[0];
    cx.ex_out = ex[1];
    run_diamond(cx, g, (int64_t)b, 1, MODE_GAP, rem);
    cluster.sync();  // keep every block's shared memory alive until its edges were read
  }
}

// status[0] = err[0] when err[0] is set (keeps an earlier error)
static __global__ void k_latch_error(const int* err, int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *err != 0 && *status == 0) *status = *err;
}

template <typename T, class Op, int P = 0, int MAXT = 1024>
__global__ void SWEPT_BOUNDS(P, MAXT) k_swept_up(Geom g, typename Op::K k, const T* u_in, T* u_out, T* e_out,
                                                   int hh, int write_top) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto cx = tiers_ctx<P>(DevCtx<T, Op>{reinterpret_cast<T*>(smraw), g, k, u_in, u_out, nullptr, e_out, Tape<T>{}});
  run_up(cx, g, (int64_t)blockIdx.x, hh, write_top != 0);
}

template <typename T, class Op, int P = 0, int MAXT = 1024>
__global__ void SWEPT_BOUNDS(P, MAXT) k_swept_diamond(Geom g, typename Op::K k, T* u_out, const T* e_in, T* e_out,
                                                        int odd, int mode, int hh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto cx = tiers_ctx<P>(DevCtx<T, Op>{reinterpret_cast<T*>(smraw), g, k, nullptr, u_out, e_in, e_out, Tape<T>{}});
  run_diamond(cx, g, (int64_t)blockIdx.x, odd, mode, hh);
}

// ---------------------------------------------------------------------------
// one slab of a grid split over ranks (Slab, swept_geom.cuh): the same pass
// phases over blocks [b0, b0 + nb), with the state at index c ul + (x - x0)
// (no wrap-around) and the edge slots of the slab's own buffers
// ---------------------------------------------------------------------------
template <typename T, class Op>
struct SlabCtx : DevCtx<T, Op> {
  static constexpr bool kSlab = true;
  Slab sl;

  __device__ __forceinline__ void load_u(int r, int c, int j, int64_t x) {
    const int64_t i = x - sl.x0;
    if (dbg::win(this->g.M, r, c, Op::C, j) && dbg::in_range(i, sl.ul, dbg::STATE))
      this->row(r, c)[j] = this->u_in[c * sl.ul + i];
  }
  __device__ __forceinline__ void store_u(int r, int c, int j, int64_t x) {
    const int64_t i = x - sl.x0;
    if (dbg::win(this->g.M, r, c, Op::C, j) && dbg::in_range(i, sl.ul, dbg::STATE))
      this->u_out[c * sl.ul + i] = this->row(r, c)[j];
  }
  __device__ __forceinline__ void load_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(this->g.M, r, c, Op::C, j) && dbg::in_range(e, slab_edge_values(this->g, sl), dbg::EDGE))
      this->row(r, c)[j] = this->e_in[e];
  }
  __device__ __forceinline__ void store_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(this->g.M, r, c, Op::C, j) && dbg::in_range(e, slab_edge_values(this->g, sl), dbg::EDGE))
      this->e_out[e] = this->row(r, c)[j];
  }
};

template <typename T, class Op, int P = 0>
__global__ void SWEPT_BOUNDS(P, 1024) k_slab_up(Geom g, Slab sl, typename Op::K k, const T* u_in, T* u_out, T* e_out,
                                                int hh, int write_top) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto cx = tiers_ctx<P>(
      SlabCtx<T, Op>{{reinterpret_cast<T*>(smraw), g, k, u_in, u_out, nullptr, e_out, Tape<T>{}}, sl});
  run_up(cx, g, sl.b0 + (int64_t)blockIdx.x, hh, write_top != 0);
}

template <typename T, class Op, int P = 0>
__global__ void SWEPT_BOUNDS(P, 1024) k_slab_diamond(Geom g, Slab sl, typename Op::K k, T* u_out, const T* e_in,
                                                     T* e_out, int odd, int mode, int hh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto cx = tiers_ctx<P>(
      SlabCtx<T, Op>{{reinterpret_cast<T*>(smraw), g, k, nullptr, u_out, e_in, e_out, Tape<T>{}}, sl});
  run_diamond(cx, g, sl.b0 + (int64_t)blockIdx.x, odd, mode, hh);
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
  static constexpr int kR = AOp::R, kC = AOp::C;
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
    if (dbg::win(g.M, r, c, kC, j)) row(r, c)[j] = u_in[c * g.N + wrap_n(x, g.N)];
  }
  __device__ __forceinline__ void store_u(int r, int c, int j, int64_t x) {
    if (dbg::win(g.M, r, c, kC, j)) u_out[c * g.N + wrap_n(x, g.N)] = row(r, c)[j];
  }
  __device__ __forceinline__ void load_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(g.M, r, c, kC, j) && dbg::in_range(e, edge_slots(g) * g.E, dbg::EDGE)) row(r, c)[j] = e_in[e];
  }
  __device__ __forceinline__ void store_edge(int r, int c, int j, int64_t e) {
    if (dbg::win(g.M, r, c, kC, j) && dbg::in_range(e, edge_slots(g) * g.E, dbg::EDGE)) e_out[e] = row(r, c)[j];
  }
  __device__ __forceinline__ void level(int s, int b, int lo, int hi, int64_t origin, int wall) {
    const int64_t L = base + b + s;
    if (dbg::level(g.M, lo, hi, kR) && dbg::ok(top - L >= 0 && top - L <= top, dbg::TAPE, L))
      adjoint_level<T, AOp>(sm, g.M, stage_c<AOp>(s), s & 1, lo, hi, wall, origin, g.N, tape + (top - L) * g.N, k,
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

// Euler classic stage: a block of B cells stages the primitives of its cells
// plus 2 halo cells per side in shared memory, computes its B + 1 face fluxes
// once (one thread each: the block has B + 32 threads), then updates its cells.
template <typename T, int STAGE>
__global__ void __launch_bounds__(288) k_classic_euler(int64_t N, int bc, typename EulerOp<T>::K k,
                                                       const T* __restrict__ in, T* out, int B) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // B cells per block; blockDim = B + 32, so each of the B + 1 faces has its own thread
  const int Wn = B + 4;
  T* pr = reinterpret_cast<T*>(smraw);
  T* pu = pr + Wn;
  T* pp = pu + Wn;
  T* F0 = pp + Wn;
  T* F1 = F0 + (B + 1);
  T* F2 = F1 + (B + 1);
  const int64_t i0 = (int64_t)blockIdx.x * B;
  for (int t = threadIdx.x; t < Wn; t += (int)blockDim.x) {
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
  for (int f = threadIdx.x; f <= B; f += (int)blockDim.x) {
    if (i0 + f > N) continue;
    typename EulerOp<T>::Prim a{pr[f], pu[f], pp[f]}, b{pr[f + 1], pu[f + 1], pp[f + 1]},
        c{pr[f + 2], pu[f + 2], pp[f + 2]}, d{pr[f + 3], pu[f + 3], pp[f + 3]};
    EulerOp<T>::flux(a, b, c, d, k, F0[f], F1[f], F2[f]);
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t i = i0 + t;
  if (t >= B || i >= N) return;
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
