// Batched swept solver: many independent heat / KS problems of different sizes
// and step counts advanced by one persistent kernel (include/swept.h,
// swept_batch_*).
//
// Work items are (problem p, pass k, tile b): the passes of each problem's
// swept launch sequence (up, diamonds, down, remainder pair; for_each_launch),
// ordered by pass layer k, then problem, then tile, so every item's
// dependencies come earlier in the order.  A persistent grid, no larger than
// the number of co-resident blocks, pulls items from one atomic counter; a
// block waits until the tiles its item reads have finished the previous pass
// (per-tile "last completed pass" counters), runs the same pass phases as the
// per-problem kernels, then publishes its own counter.  Every wait is bounded:
// past the limit the block records SWEPT_ETIMEOUT in the error word and stops.
//
// Hazards.  A diamond of pass k at tile b reads the edges of tiles l(b), r(b)
// written in pass k-1 (buffer (k-1)&1) and writes its own to buffer k&1.  The
// blocks that read tile b's pass-(k-2) edges from buffer k&1 are exactly l(b)
// and r(b) of pass k-1 (the zig-zag makes the reader set of pass k-1 equal the
// dependency set of pass k), so waiting for them also protects the buffer
// from being overwritten early.  The remainder trapezoid of tile b waits for
// tiles b-1, b, b+1 of the down pass (which wrote its part of the state), the
// gap pass for trapezoids b and b+1.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "debug_check.cuh"
#include "impl.h"
#include "kernels.cuh"
#include "ops.cuh"
#include "swept.h"
#include "trace.h"
#include "swept_phases.cuh"

namespace swept {
namespace {

struct BatchProb {
  int64_t n, nt;
  int64_t u_off;   // first value of this problem in the state array
  int64_t e_off;   // first value of this problem's two edge buffers
  int64_t t0;      // first tile counter of this problem
  int64_t cblk0;   // first block of this problem in the classic launches
  int64_t n_sub;   // sub-timesteps (nsteps * S)
  int32_t kind;    // SWEPT_HEAT / SWEPT_KS
  int32_t W, h, R, S;
  int32_t q, rem, npass;
  int32_t pad;
  alignas(16) unsigned char k[KBYTES];
};

struct BatchDev {
  const BatchProb* probs;
  const int64_t* gstart;  // item index where group g starts (G + 1 entries)
  const int32_t* gprob;
  const int32_t* gpass;
  int32_t ngroups;
  int64_t total;
  int64_t start_item;     // items before it are treated as never scheduled (fault tests)
  int* done;              // last completed pass per tile
  unsigned long long* queue;
  int* error;
  uint32_t spin_limit;
};

// Block context of one item: like the per-problem DevCtx, but global reads
// go through L2 (ld.global.cg) because other SMs write these buffers while
// this persistent block runs and L1 is not coherent.
template <typename T, class Op>
struct BatchCtx {
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
  // the per-problem kernels' tier code (strided, or paired for radius 2)
  __device__ __forceinline__ void level(int s, int, int lo, int hi, int64_t, int wall) {
    if (dbg::level(g.M, lo, hi, kR)) LevelImpl<T, Op>::run(sm, g.M, stage_c<Op>(s), s & 1, lo, hi, wall, 1, k);
    __syncthreads();
  }
};

__device__ __forceinline__ Geom geom_of(const BatchProb& p) {
  Geom g;
  g.N = p.n;
  g.nt = p.nt;
  g.W = p.W;
  g.R = p.R;
  g.S = p.S;
  g.C = 1;
  g.h = p.h;
  g.M = p.W + 2 * p.R;
  g.E = 2 * p.h * 2 * p.R;
  g.bc = 0;
  g.chunk = 1;
  return g;
}

// bounded wait for *flag >= need; gives up at the limit or once another block
// has recorded an error
__device__ __forceinline__ bool wait_ge(const int* flag, int need, uint32_t limit, const int* error) {
  for (uint32_t i = 0;; ++i) {
    if (*(volatile const int*)flag >= need) return true;
    if (i >= limit || *(volatile const int*)error != 0) return false;
    __nanosleep(128);
  }
}

// thread 0: wait for the item's inputs; false on timeout
__device__ bool wait_inputs(const BatchDev& d, const BatchProb& p, int k, int64_t b) {
  // the single-problem persistent kernel's rule (persist_deps), per problem
  const int* done = d.done + p.t0;
  int64_t tile[3];
  int need[3];
  const int n = persist_deps(geom_of(p), (int64_t)p.q * p.h + p.rem, k, b, tile, need);
  for (int i = 0; i < n; ++i)
    if (!dbg::in_range(tile[i], p.nt, dbg::COUNTER) || !wait_ge(done + tile[i], need[i], d.spin_limit, d.error))
      return false;
  return true;
}

template <typename T, class Op>
__device__ void run_item(T* sm, const BatchProb& p, int k, int64_t b, T* u_all, T* e_all) {
  BatchCtx<T, Op> cx;
  cx.sm = sm;
  cx.g = geom_of(p);
  memcpy(&cx.k, p.k, sizeof(cx.k));
  cx.u = u_all + p.u_off;
  T* eb[2] = {e_all + p.e_off, e_all + p.e_off + p.nt * (int64_t)cx.g.E};
  const int main_passes = p.q > 0 ? p.q + 1 : 0;
  if (k < main_passes) {
    if (k == 0) {
      cx.e_in = nullptr;
      cx.e_out = eb[0];
      run_up(cx, cx.g, b, p.h, false);
    } else {
      cx.e_in = eb[(k - 1) & 1];
      cx.e_out = eb[k & 1];
      run_diamond(cx, cx.g, b, k & 1, k == p.q ? MODE_DOWN : MODE_DIAMOND, p.h);
    }
  } else if (k == main_passes) {
    cx.e_in = nullptr;
    cx.e_out = eb[0];
    run_up(cx, cx.g, b, p.rem, true);
  } else {
    cx.e_in = eb[0];
    cx.e_out = eb[1];
    run_diamond(cx, cx.g, b, 1, MODE_GAP, p.rem);
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_batch(BatchDev d, T* u_all, T* e_all) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int64_t s_item;
  __shared__ int s_ok;
  T* sm = reinterpret_cast<T*>(smraw);
  for (;;) {
    if (threadIdx.x == 0) s_item = d.start_item + (int64_t)atomicAdd(d.queue, 1ULL);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= d.total) break;
    // group of the item (binary search on gstart)
    int lo = 0, hi = d.ngroups - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d.gstart[mid] <= item)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BatchProb& p = d.probs[d.gprob[lo]];
    const int k = d.gpass[lo];
    const int64_t b = item - d.gstart[lo];
    if (threadIdx.x == 0) {
      s_ok = (*(volatile int*)d.error == 0) && wait_inputs(d, p, k, b);
      if (!s_ok) atomicCAS(d.error, 0, (int)SWEPT_ETIMEOUT);
      __threadfence();
    }
    __syncthreads();
    if (!s_ok) break;
    if (p.kind == SWEPT_HEAT)
      run_item<T, HeatOp<T>>(sm, p, k, b, u_all, e_all);
    else
      run_item<T, KsOp<T>>(sm, p, k, b, u_all, e_all);
    __threadfence();  // every thread's edge / state writes visible device-wide ...
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(d.done + p.t0 + b, k);  // ... before the tile is published
  }
}

// ---------------------------------------------------------------------------
// Classic decomposition of a batch (the baseline of the batched swept solver):
// launch k advances every problem that still has a sub-timestep k, one point
// per thread, through global memory (Section "Classic scheme"), with the same
// per-point operation as classic_step_n.  Problems are ordered by sub-timestep
// count, longest first, so the active problems of launch k are a prefix and
// the launch covers the blocks [0, cblk(k)).  kBatchClassicBlock points per
// block, each block inside one problem (blk_prob).  A heat problem alternates
// u -> tmp (even k) and tmp -> u (odd k); a KS problem runs stage k mod 2:
// u -> tmp (predictor), then tmp, u -> u.
// ---------------------------------------------------------------------------
constexpr int kBatchClassicBlock = 256;

template <typename T, class Op, int STAGE>
__device__ __forceinline__ void classic_point(const BatchProb& p, int64_t i, const T* in, T* out) {
  constexpr int R = Op::R;
  typename Op::K k;
  memcpy(&k, p.k, sizeof(k));
  T v[2 * R + 1];
  if (i >= R && i < p.n - R) {
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) v[d] = in[i + d - R];
  } else {
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) v[d] = in[wrap_n(i + d - R, p.n)];
  }
  const T p2 = STAGE == 1 ? out[i] : T(0);
  out[i] = Op::template point<STAGE>(v, p2, k);
}

template <typename T>
__global__ void __launch_bounds__(kBatchClassicBlock) k_classic_batch(const BatchProb* probs, const int32_t* blk_prob,
                                                                      int64_t k, T* u_all, T* t_all) {
  const BatchProb& p = probs[blk_prob[blockIdx.x]];
  const int64_t i = ((int64_t)blockIdx.x - p.cblk0) * kBatchClassicBlock + threadIdx.x;
  if (i >= p.n) return;
  T* u = u_all + p.u_off;
  T* t = t_all + p.u_off;
  if (p.kind == SWEPT_HEAT) {
    if ((k & 1) == 0)
      classic_point<T, HeatOp<T>, 0>(p, i, u, t);
    else
      classic_point<T, HeatOp<T>, 0>(p, i, t, u);
  } else {
    if ((k & 1) == 0)
      classic_point<T, KsOp<T>, 0>(p, i, u, t);
    else
      classic_point<T, KsOp<T>, 1>(p, i, t, u);
  }
}

// a heat problem with an odd sub-timestep count ends in tmp: copy it back
template <typename T>
__global__ void __launch_bounds__(kBatchClassicBlock) k_classic_batch_finish(const BatchProb* probs,
                                                                             const int32_t* blk_prob, T* u_all,
                                                                             const T* t_all) {
  const BatchProb& p = probs[blk_prob[blockIdx.x]];
  if (p.kind != SWEPT_HEAT || (p.n_sub & 1) == 0) return;
  const int64_t i = ((int64_t)blockIdx.x - p.cblk0) * kBatchClassicBlock + threadIdx.x;
  if (i < p.n) u_all[p.u_off + i] = t_all[p.u_off + i];
}

}  // namespace
}  // namespace swept

using swept::BatchProb;

struct swept_batch {
  int dtype = 0;
  int threads = 0;
  size_t smem = 0;
  int device = -1;
  int sm_count = 0;
  std::vector<BatchProb> probs;
  std::vector<int64_t> gstart;
  std::vector<int32_t> gprob, gpass;
  std::vector<int64_t> offsets;
  int64_t total_items = 0, total_tiles = 0, state_values = 0, edge_values = 0;
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0, ws_bound = 0;
  size_t off_probs = 0, off_gstart = 0, off_gprob = 0, off_gpass = 0, off_done = 0, off_ctl = 0, off_edges = 0;
  int grid = 0;
  int64_t start_item = 0;
  uint32_t spin_limit = 1u << 24;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* exec_u = nullptr;
  // classic baseline: blocks of launch k are [0, cblk_end[k]) (problems sorted
  // by sub-timestep count, longest first); graphs of kClassicChunk launches
  std::vector<int32_t> blk_prob;
  std::vector<int64_t> cblk_end;
  int64_t max_sub = 0;
  size_t off_blk = 0, off_tmp = 0;
  std::vector<cudaGraphExec_t> cexec;
  const void* cexec_u = nullptr;
  std::string err;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

swept_status bfail(swept_batch* b, swept_status st, const std::string& m) {
  if (b) b->err = m;
  return st;
}

void drop_graph(swept_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->exec_u = nullptr;
  for (cudaGraphExec_t x : b->cexec) cudaGraphExecDestroy(x);
  b->cexec.clear();
  b->cexec_u = nullptr;
}

constexpr int64_t kClassicChunk = 1024;  // classic launches per captured graph

// classic launches [k0, k1) of the batch (and the final copy when k1 is the end)
cudaError_t launch_classic(swept_batch* b, void* u, int64_t k0, int64_t k1, cudaStream_t s) {
  const BatchProb* probs = (const BatchProb*)(b->ws + b->off_probs);
  const int32_t* bp = (const int32_t*)(b->ws + b->off_blk);
  for (int64_t k = k0; k < k1; ++k) {
    const unsigned grid = (unsigned)b->cblk_end[(size_t)k];
    if (b->dtype == SWEPT_F64)
      swept::k_classic_batch<double><<<grid, swept::kBatchClassicBlock, 0, s>>>(probs, bp, k, (double*)u,
                                                                                (double*)(b->ws + b->off_tmp));
    else
      swept::k_classic_batch<float><<<grid, swept::kBatchClassicBlock, 0, s>>>(probs, bp, k, (float*)u,
                                                                               (float*)(b->ws + b->off_tmp));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (k1 == b->max_sub && !b->blk_prob.empty()) {
    const unsigned grid = (unsigned)b->blk_prob.size();
    if (b->dtype == SWEPT_F64)
      swept::k_classic_batch_finish<double><<<grid, swept::kBatchClassicBlock, 0, s>>>(
          probs, bp, (double*)u, (const double*)(b->ws + b->off_tmp));
    else
      swept::k_classic_batch_finish<float><<<grid, swept::kBatchClassicBlock, 0, s>>>(
          probs, bp, (float*)u, (const float*)(b->ws + b->off_tmp));
    return cudaGetLastError();
  }
  return cudaSuccess;
}

int default_batch_tile(int64_t n, int R) {
  for (int W = 512; W >= 4 * R; W /= 2)
    if (n % W == 0 && n / W >= 2 && W % (4 * R) == 0) return W;
  return 0;
}

cudaError_t launch_batch(swept_batch* b, void* u, cudaStream_t s) {
  char* ws = b->ws;
  cudaError_t e = cudaMemsetAsync(ws + b->off_done, 0xFF, (size_t)b->total_tiles * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + b->off_ctl, 0, kAlign, s);
  if (e != cudaSuccess) return e;
  swept::BatchDev d;
  d.probs = (const BatchProb*)(ws + b->off_probs);
  d.gstart = (const int64_t*)(ws + b->off_gstart);
  d.gprob = (const int32_t*)(ws + b->off_gprob);
  d.gpass = (const int32_t*)(ws + b->off_gpass);
  d.ngroups = (int32_t)b->gprob.size();
  d.total = b->total_items;
  d.start_item = b->start_item;
  d.done = (int*)(ws + b->off_done);
  d.queue = (unsigned long long*)(ws + b->off_ctl);
  d.error = (int*)(ws + b->off_ctl + 64);
  d.spin_limit = b->spin_limit;
  if (b->dtype == SWEPT_F64)
    swept::k_batch<double><<<b->grid, b->threads, b->smem, s>>>(d, (double*)u, (double*)(ws + b->off_edges));
  else
    swept::k_batch<float><<<b->grid, b->threads, b->smem, s>>>(d, (float*)u, (float*)(ws + b->off_edges));
  return cudaGetLastError();
}

}  // namespace

extern "C" {

swept_status swept_batch_plan(const swept_batch_problem* problems, int64_t count, int32_t dtype, int32_t threads,
                              swept_batch** out) {
  if (!problems || count <= 0 || !out || (dtype != SWEPT_F32 && dtype != SWEPT_F64)) return SWEPT_EINVAL;
  *out = nullptr;
  swept_batch* b = new (std::nothrow) swept_batch();
  if (!b) return SWEPT_EINVAL;
  b->dtype = dtype;
  const size_t vb = dtype == SWEPT_F64 ? 8 : 4;
  int maxM = 0, maxR = 1;
  int64_t u_off = 0, e_off = 0, t0 = 0;
  b->probs.resize((size_t)count);
  b->offsets.resize((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    const swept_batch_problem& q = problems[i];
    const swept::SchemeImpl* im = q.scheme == SWEPT_HEAT ? swept::heat_impl(dtype)
                                  : q.scheme == SWEPT_KS ? swept::ks_impl(dtype)
                                                         : nullptr;
    if (!im || q.nsteps < 0 || q.n < 8 || !(q.dx > 0) || !(q.dt > 0)) {
      delete b;
      return SWEPT_EINVAL;
    }
    const int R = im->R;
    const int W = q.tile_w > 0 ? q.tile_w : default_batch_tile(q.n, R);
    if (W < 4 * R || W % (4 * R) != 0 || q.n % W != 0 || q.n / W < 2) {
      delete b;
      return SWEPT_EINVAL;
    }
    BatchProb& p = b->probs[(size_t)i];
    memset(&p, 0, sizeof(p));
    p.n = q.n;
    p.nt = q.n / W;
    p.kind = q.scheme;
    p.W = W;
    p.R = R;
    p.S = im->S;
    p.h = W / (2 * R);
    const int64_t n_sub = q.nsteps * p.S;
    p.q = (int32_t)(n_sub / p.h);
    p.rem = (int32_t)(n_sub % p.h);
    p.npass = (p.q > 0 ? p.q + 1 : 0) + (p.rem > 0 ? 2 : 0);
    double param[4] = {q.param, 0, 0, 0};
    im->make_consts(param, q.dx, q.dt, p.k);
    p.u_off = u_off;
    b->offsets[(size_t)i] = u_off;
    u_off += (q.n + 63) / 64 * 64;  // 256-byte aligned starts in FP32 and FP64
    p.n_sub = n_sub;
    p.e_off = e_off;
    e_off += 2 * p.nt * (int64_t)(2 * p.h * 2 * R);
    p.t0 = t0;
    t0 += p.nt;
    maxM = std::max(maxM, W + 2 * R);
    maxR = std::max(maxR, R);
  }
  b->state_values = u_off;
  b->edge_values = e_off;
  b->total_tiles = t0;
  // classic baseline: problems by sub-timestep count, longest first; each
  // problem's points in whole blocks of kBatchClassicBlock
  {
    std::vector<int64_t> order((size_t)count);
    for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
      return b->probs[(size_t)a].n_sub > b->probs[(size_t)c].n_sub;
    });
    b->max_sub = b->probs[(size_t)order[0]].n_sub;
    b->cblk_end.assign((size_t)b->max_sub, 0);
    int64_t blk = 0;
    for (int64_t j = 0; j < count; ++j) {
      BatchProb& p = b->probs[(size_t)order[(size_t)j]];
      p.cblk0 = blk;
      const int64_t nb = (p.n + swept::kBatchClassicBlock - 1) / swept::kBatchClassicBlock;
      for (int64_t x = 0; x < nb; ++x) b->blk_prob.push_back((int32_t)order[(size_t)j]);
      blk += nb;
      // launches k < n_sub of this problem cover its blocks (the prefix grows)
      for (int64_t k = 0; k < p.n_sub; ++k) b->cblk_end[(size_t)k] = blk;
    }
  }
  // groups: layer k, problem p, with nt_p items each
  int maxpass = 0;
  for (auto& p : b->probs) maxpass = std::max(maxpass, (int)p.npass);
  int64_t item = 0;
  for (int k = 0; k < maxpass; ++k)
    for (int64_t i = 0; i < count; ++i)
      if (b->probs[(size_t)i].npass > k) {
        b->gstart.push_back(item);
        b->gprob.push_back((int32_t)i);
        b->gpass.push_back(k);
        item += b->probs[(size_t)i].nt;
      }
  b->total_items = item;
  b->gstart.push_back(item);
  if (b->gprob.empty()) b->gprob.push_back(0), b->gpass.push_back(0);
  b->threads = threads > 0 ? threads : 256;
  if (b->threads < 32 || b->threads > 1024 || b->threads % 32) {
    delete b;
    return SWEPT_EINVAL;
  }
  b->smem = (size_t)2 * maxM * vb;
  // workspace layout
  size_t off = 0;
  b->off_probs = off;
  off = align_up(off + b->probs.size() * sizeof(BatchProb));
  b->off_gstart = off;
  off = align_up(off + b->gstart.size() * sizeof(int64_t));
  b->off_gprob = off;
  off = align_up(off + b->gprob.size() * sizeof(int32_t));
  b->off_gpass = off;
  off = align_up(off + b->gpass.size() * sizeof(int32_t));
  b->off_done = off;
  off = align_up(off + (size_t)b->total_tiles * sizeof(int));
  b->off_ctl = off;
  off += kAlign;
  b->off_edges = off;
  off = align_up(off + (size_t)b->edge_values * vb);
  b->off_blk = off;
  off = align_up(off + b->blk_prob.size() * sizeof(int32_t));
  b->off_tmp = off;
  off = align_up(off + (size_t)b->state_values * vb);
  b->ws_bytes = off;
  int dev = -1;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      b->device = dev;
      b->sm_count = sms;
    }
  }
  cudaGetLastError();
  *out = b;
  return SWEPT_OK;
}

swept_status swept_batch_sizes(const swept_batch* b, int64_t* offsets, int64_t* state_values, size_t* ws_bytes,
                               int64_t* items) {
  if (!b) return SWEPT_EINVAL;
  if (offsets) memcpy(offsets, b->offsets.data(), b->offsets.size() * sizeof(int64_t));
  if (state_values) *state_values = b->state_values;
  if (ws_bytes) *ws_bytes = b->ws_bytes;
  if (items) *items = b->total_items;
  return SWEPT_OK;
}

swept_status swept_batch_bind_workspace(swept_batch* b, void* ws_dev, size_t bytes) {
  if (!b) return SWEPT_EINVAL;
  if (!ws_dev || ((uintptr_t)ws_dev % kAlign) != 0) return bfail(b, SWEPT_EINVAL, "workspace NULL or misaligned");
  if (bytes < b->ws_bytes) return bfail(b, SWEPT_ENOMEM_WORKSPACE, "workspace too small");
  if (b->device < 0) return bfail(b, SWEPT_ECUDA, "no CUDA device");
  drop_graph(b);
  b->ws = (char*)ws_dev;
  b->ws_bound = bytes;
  cudaError_t e = cudaMemcpy(b->ws + b->off_probs, b->probs.data(), b->probs.size() * sizeof(BatchProb),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->ws + b->off_gstart, b->gstart.data(), b->gstart.size() * sizeof(int64_t),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->ws + b->off_gprob, b->gprob.data(), b->gprob.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->ws + b->off_gpass, b->gpass.data(), b->gpass.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->blk_prob.empty())
    e = cudaMemcpy(b->ws + b->off_blk, b->blk_prob.data(), b->blk_prob.size() * sizeof(int32_t),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
  // persistent grid: at most the co-resident blocks
  const void* fn = b->dtype == SWEPT_F64 ? (const void*)swept::k_batch<double> : (const void*)swept::k_batch<float>;
  e = swept::raise_smem_limit(fn, b->smem);
  if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "shared-memory limit");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, b->threads, b->smem);
  if (e != cudaSuccess || per_sm < 1) return bfail(b, SWEPT_EINVAL, "batch kernel does not fit on an SM");
  b->grid = (int)std::min<int64_t>(std::max<int64_t>(1, b->total_items), (int64_t)per_sm * b->sm_count);
  if (!b->cap) {
    e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "stream");
  }
  return SWEPT_OK;
}

swept_status swept_batch_set_option(swept_batch* b, int32_t option, int64_t value) {
  if (!b) return SWEPT_EINVAL;
  if (option == SWEPT_BATCH_SPIN_LIMIT && value > 0 && value <= 0xffffffffLL) {
    b->spin_limit = (uint32_t)value;
  } else if (option == SWEPT_BATCH_START_ITEM && value >= 0) {
    b->start_item = value;
  } else if (option == SWEPT_BATCH_GRID && value >= 0) {
    if (value > 0 && b->grid > 0) b->grid = (int)std::min<int64_t>(value, b->grid);
  } else {
    return bfail(b, SWEPT_EINVAL, "unknown option or value");
  }
  drop_graph(b);
  return SWEPT_OK;
}

swept_status swept_batch_run(swept_batch* b, void* u_dev, void* stream) {
  const swept_trace::Range trace_range("swept_batch_run");
  if (!b || !u_dev) return SWEPT_EINVAL;
  if (!b->ws) return bfail(b, SWEPT_ENOWORKSPACE, "no workspace bound");
  if (b->total_items == 0) return SWEPT_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) {
    e = launch_batch(b, u_dev, s);
    return e == cudaSuccess ? SWEPT_OK : bfail(b, SWEPT_ECUDA, cudaGetErrorString(e));
  }
  if (!b->exec || b->exec_u != u_dev) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->exec_u = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "begin capture");
    cudaError_t le = launch_batch(b, u_dev, b->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, SWEPT_ECUDA, cudaGetErrorString(le != cudaSuccess ? le : e));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "graph instantiate");
    b->exec_u = u_dev;
  }
  e = cudaGraphLaunch(b->exec, s);
  return e == cudaSuccess ? SWEPT_OK : bfail(b, SWEPT_ECUDA, cudaGetErrorString(e));
}

swept_status swept_batch_run_classic(swept_batch* b, void* u_dev, void* stream) {
  const swept_trace::Range trace_range("swept_batch_run_classic");
  if (!b || !u_dev) return SWEPT_EINVAL;
  if (!b->ws) return bfail(b, SWEPT_ENOWORKSPACE, "no workspace bound");
  if (b->max_sub == 0) return SWEPT_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) {
    e = launch_classic(b, u_dev, 0, b->max_sub, s);
    return e == cudaSuccess ? SWEPT_OK : bfail(b, SWEPT_ECUDA, cudaGetErrorString(e));
  }
  if (b->cexec.empty() || b->cexec_u != u_dev) {
    for (cudaGraphExec_t x : b->cexec) cudaGraphExecDestroy(x);
    b->cexec.clear();
    for (int64_t k0 = 0; k0 < b->max_sub; k0 += kClassicChunk) {
      const int64_t k1 = std::min(b->max_sub, k0 + kClassicChunk);
      e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "begin capture");
      const cudaError_t le = launch_classic(b, u_dev, k0, k1, b->cap);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(b->cap, &g);
      if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, SWEPT_ECUDA, cudaGetErrorString(le != cudaSuccess ? le : e));
      }
      cudaGraphExec_t x = nullptr;
      e = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, "graph instantiate");
      b->cexec.push_back(x);
    }
    b->cexec_u = u_dev;
  }
  for (cudaGraphExec_t x : b->cexec) {
    e = cudaGraphLaunch(x, s);
    if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, cudaGetErrorString(e));
  }
  return SWEPT_OK;
}

swept_status swept_batch_sync_status(swept_batch* b, void* stream) {
  if (!b || !b->ws) return SWEPT_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  int word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, b->ws + b->off_ctl + 64, sizeof word, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bfail(b, SWEPT_ECUDA, cudaGetErrorString(e));
  if (word == 0) return SWEPT_OK;
  return bfail(b, word == SWEPT_ETIMEOUT ? SWEPT_ETIMEOUT : SWEPT_EDEVICE, "device-side error word set");
}

swept_status swept_batch_last_error(const swept_batch* b, char* buf, size_t len) {
  if (!b || !buf || len == 0) return SWEPT_EINVAL;
  snprintf(buf, len, "%s", b->err.c_str());
  return SWEPT_OK;
}

void swept_batch_free(swept_batch* b) {
  if (!b) return;
  drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

}  // extern "C"
