// C-ABI runtime: plan selection, workspace layout, launch sequencing of the
// swept and classic paths, and CUDA-graph caching (include/swept.h).
#include <stdio.h>
#include <string.h>

#include <functional>
#include <new>
#include <string>
#include <vector>

#include <algorithm>
#include <mutex>

#include "graph_cache.h"
#include "kernels.cuh"
#include "runtime.h"
#include "trace.h"
#include "swept_phases.cuh"

using swept::Geom;
using swept::SchemeImpl;

namespace {

constexpr size_t kAlign = 256;
constexpr int kGb300Sms = 152;
constexpr int kGb300SmemOptin = 232448;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

swept_status fail(swept_handle* h, swept_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}
swept_status cuda_fail(swept_handle* h, cudaError_t e, const char* where) {
  return fail(h, SWEPT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

const SchemeImpl* pick_impl(int scheme, int dtype) {
  if (dtype != SWEPT_F32 && dtype != SWEPT_F64) return nullptr;
  switch (scheme) {
    case SWEPT_HEAT: return swept::heat_impl(dtype);
    case SWEPT_KS: return swept::ks_impl(dtype);
    case SWEPT_EULER: return swept::euler_impl(dtype);
    default: return nullptr;
  }
}

// A tile width is legal when it is a multiple of 4R (so the half cycle h =
// W/(2R) is even and the tips meet at whole points) and the grid holds at
// least two tiles; a grid that is not a multiple of W gets a wider last tile.
bool tile_ok(int64_t n, int W, int R) { return W >= 4 * R && W % (4 * R) == 0 && n / W >= 2; }
bool tile_divides(int64_t n, int W, int R) { return tile_ok(n, W, R) && n % W == 0; }

// Default tile width: the largest W <= 1024 (multiple of 4R, dividing n) that
// still gives at least two blocks per SM; else at least one per SM; else the
// smallest such W.  When no multiple of 4R divides n, the same rules choose
// among all legal widths (the last tile then carries the n mod W extra points).
int choose_tile(int64_t n, int R, int sms) {
  for (int pass = 0; pass < 2; ++pass) {
    auto ok = [&](int W) { return pass == 0 ? tile_divides(n, W, R) : tile_ok(n, W, R); };
    int best = 0;
    for (int W = 4 * R; W <= 1024; W += 4 * R)
      if (ok(W) && n / W >= 2 * sms) best = W;
    if (best) return best;
    for (int W = 4 * R; W <= 1024; W += 4 * R)
      if (ok(W) && n / W >= sms) best = W;
    if (best) return best;
    for (int W = 4 * R; W <= 4096; W += 4 * R)
      if (ok(W)) return W;
  }
  return 0;
}

swept_status no_tiling(swept_handle* h) {
  return fail(h, SWEPT_EUNSUPPORTED, "grid too small for a swept tiling (fewer than two tiles of 4r points): "
                                     "only classic_step_n runs on this handle");
}


swept_status run_graph(swept_handle* h, const std::string& key, cudaStream_t user,
                       const std::function<cudaError_t(cudaStream_t)>& issue) {
  return swept_graphs::run(h, key, user, issue);
}
void drop_graphs(swept_handle* h) { swept_graphs::drop(h); }
using swept_graphs::key_of;

// First GPU use of a handle: the private capture stream and the shared-memory
// limit of the swept kernels.  Later calls check the current device matches.
swept_status ensure_device(swept_handle* h) {
  if (h->device < 0) return fail(h, SWEPT_ECUDA, "no CUDA device was available when the handle was created");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
  if (dev != h->device) return fail(h, SWEPT_EINVAL, "current device differs from the handle's device");
  if (!h->cap) {
    if (h->smem > 48 * 1024) {
      e = h->impl->prepare(h->smem);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
    }
    e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreateWithFlags");
  }
  return SWEPT_OK;
}

swept_status check_ready(swept_handle* h, void* u_dev, int64_t nsteps) {
  if (!h) return SWEPT_EINVAL;
  if (!u_dev || nsteps < 0) return fail(h, SWEPT_EINVAL, "u_dev is NULL or nsteps < 0");
  if (!h->ws) return fail(h, SWEPT_ENOWORKSPACE, "no workspace bound (swept_bind_workspace)");
  if (h->ws_bound < h->ws_bytes) return fail(h, SWEPT_ENOMEM_WORKSPACE, "bound workspace too small");
  return ensure_device(h);
}

// ---------------------------------------------------------------------------
// swept launch sequence: launch index i in [from, to) of for_each_launch
// ---------------------------------------------------------------------------
cudaError_t issue_swept(swept_handle* h, void* u, int64_t n_sub, int64_t from, int64_t to, cudaStream_t s) {
  const Geom& g = h->g;
  const SchemeImpl* im = h->impl;
  void* eb[2] = {h->ws + h->off_e0, h->ws + h->off_e1};
  int64_t idx = 0;
  cudaError_t err = cudaSuccess;
  swept::for_each_launch(g, n_sub, [&](int kind, int odd, int mode, int hh, int64_t pass) {
    const int64_t i = idx++;
    if (i < from || i >= to || err != cudaSuccess) return;
    if (kind == 0) {
      const int out = pass >= 0 ? (int)(pass & 1) : 0;
      err = im->up(g, h->k, u, u, eb[out], hh, mode == swept::MODE_GAP, h->threads, h->smem, s);
    } else {
      const int in = pass >= 1 ? (int)((pass - 1) & 1) : 0;
      const int out = pass >= 1 ? (int)(pass & 1) : 1;
      err = im->diamond(g, h->k, u, eb[in], eb[out], odd, mode, hh, h->threads, h->smem, s);
    }
  });
  return err;
}

int64_t swept_launch_count(const Geom& g, int64_t n_sub) {
  const int64_t q = n_sub / g.h, rem = n_sub % g.h;
  return (q > 0 ? q + 1 : 0) + (rem > 0 ? 2 : 0);
}

// classic sub-timesteps [k0, k1) of a run; for a one-stage scheme the state
// ping-pongs between u (even k) and tmp (odd k)
cudaError_t issue_classic(swept_handle* h, void* u, int64_t k0, int64_t k1, cudaStream_t s) {
  const Geom& g = h->g;
  void* tmp = h->ws + h->off_tmp;
  for (int64_t k = k0; k < k1; ++k) {
    cudaError_t e;
    if (g.S == 1) {
      const bool even = (k & 1) == 0;
      e = h->impl->classic(g, h->k, 0, even ? u : tmp, even ? tmp : u, s);
    } else {
      const int stage = (int)(k % g.S);
      e = stage == 0 ? h->impl->classic(g, h->k, 0, u, tmp, s) : h->impl->classic(g, h->k, 1, tmp, u, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// adjoint support: checkpoint layout, tape-recording forward, adjoint sweep
// ---------------------------------------------------------------------------
struct AdjPlan {
  int64_t K = 0, nseg = 0;
  size_t off_ck = 0, off_tape = 0, off_lam = 0, off_w = 0, off_slots = 0, bytes = 0;
};

AdjPlan adj_layout(const swept_handle* h, int64_t nsteps, int64_t K) {
  AdjPlan a;
  const size_t slot = align_up((size_t)h->g.N * h->g.C * sizeof(double));
  a.K = K;
  a.nseg = (nsteps + K - 1) / K;
  a.off_ck = 0;
  a.off_tape = a.off_ck + (size_t)a.nseg * slot;
  // the tape's tiers are contiguous runs of N*C values (the kernels index them so)
  a.off_lam = a.off_tape + align_up((size_t)(h->g.S * K + 1) * h->g.N * h->g.C * sizeof(double));
  a.off_w = a.off_lam + slot;
  a.off_slots = a.off_w + slot;
  a.bytes = a.off_slots + align_up((size_t)2 * h->g.nt * sizeof(double));  // (hi, lo) per block
  return a;
}

// steps per segment: whole passes (h/S steps) or the whole run.  For a size
// query (bytes == 0) the segment that needs the least memory: the buffer holds
// ceil(nsteps / K) checkpoints plus a tape of S K + 1 tiers, smallest near
// K = sqrt(nsteps / S), and every choice recomputes each step once.  Otherwise
// the largest segment that fits `bytes`.
int64_t adj_segment(const swept_handle* h, int64_t nsteps, size_t bytes) {
  const int64_t K0 = h->g.h / h->g.S;
  if (nsteps <= K0) return nsteps;
  if (bytes == 0) {
    int64_t best = nsteps;
    size_t best_bytes = adj_layout(h, nsteps, nsteps).bytes;
    for (int64_t K = K0; K < nsteps; K += K0) {
      const size_t b = adj_layout(h, nsteps, K).bytes;
      if (b < best_bytes) best = K, best_bytes = b;
    }
    return best;
  }
  if (adj_layout(h, nsteps, nsteps).bytes <= bytes) return nsteps;
  for (int64_t K = (nsteps / K0) * K0; K >= K0; K -= K0)
    if (adj_layout(h, nsteps, K).bytes <= bytes) return K;
  return 0;
}

int64_t launch_base(const Geom& g, int64_t n_sub, int kind, int64_t pass) {
  const int64_t q = n_sub / g.h;
  return pass >= 0 ? (kind == 0 ? 0 : (pass - 1) * (int64_t)g.h) : q * (int64_t)g.h;
}

size_t adj_smem(const swept_handle* h) { return std::max<size_t>(h->smem, 64 * sizeof(double)); }

// swept forward over n_sub sub-timesteps of u, recording tier L (1..n_sub) into
// tape slot L (N*C values per slot, slot 0 = the starting state, copied by the caller)
cudaError_t issue_swept_tape(swept_handle* h, void* u, int64_t n_sub, void* tape, cudaStream_t s) {
  const Geom& g = h->g;
  const SchemeImpl* im = h->impl;
  void* eb[2] = {h->ws + h->off_e0, h->ws + h->off_e1};
  cudaError_t err = cudaSuccess;
  swept::for_each_launch(g, n_sub, [&](int kind, int odd, int mode, int hh, int64_t pass) {
    if (err != cudaSuccess) return;
    const int64_t base = launch_base(g, n_sub, kind, pass);
    if (kind == 0) {
      const int out = pass >= 0 ? (int)(pass & 1) : 0;
      err = im->up_tape(g, h->k, u, u, eb[out], hh, mode == swept::MODE_GAP, h->threads, h->smem, tape, 0,
                        n_sub + 1, base, s);
    } else {
      const int in = pass >= 1 ? (int)((pass - 1) & 1) : 0;
      const int out = pass >= 1 ? (int)(pass & 1) : 1;
      err = im->diamond_tape(g, h->k, u, eb[in], eb[out], odd, mode, hh, h->threads, h->smem, tape, 0, n_sub + 1,
                             base, s);
    }
  });
  return err;
}

// adjoint sweep of lam over n_sub reverse sub-timesteps against tape slots n_sub..0
cudaError_t issue_adjoint(swept_handle* h, const void* ka, void* lam, int64_t n_sub, const void* tape, double* slots,
                          cudaStream_t s) {
  const Geom& g = h->g;
  const SchemeImpl* im = h->impl;
  void* eb[2] = {h->ws + h->off_e0, h->ws + h->off_e1};
  const size_t sm = adj_smem(h);
  cudaError_t err = cudaSuccess;
  swept::for_each_launch(g, n_sub, [&](int kind, int odd, int mode, int hh, int64_t pass) {
    if (err != cudaSuccess) return;
    const int64_t base = launch_base(g, n_sub, kind, pass);
    if (kind == 0) {
      const int out = pass >= 0 ? (int)(pass & 1) : 0;
      err = im->adj_up(g, ka, lam, lam, eb[out], hh, mode == swept::MODE_GAP, h->threads, sm, tape, n_sub, base,
                       slots, s);
    } else {
      const int in = pass >= 1 ? (int)((pass - 1) & 1) : 0;
      const int out = pass >= 1 ? (int)(pass & 1) : 1;
      err = im->adj_diamond(g, ka, lam, eb[in], eb[out], odd, mode, hh, h->threads, sm, tape, n_sub, base, slots, s);
    }
  });
  return err;
}

swept_status adj_check(swept_handle* h, int64_t nsteps, void* ckpt, size_t bytes, AdjPlan* plan) {
  if (!h->impl->adj_up || h->cfg.dtype != SWEPT_F64)
    return fail(h, SWEPT_EUNSUPPORTED, "the adjoint exists for heat and KS in FP64 only");
  if (!h->tiled) return no_tiling(h);
  if (!ckpt || nsteps < 0 || ((uintptr_t)ckpt % kAlign) != 0)
    return fail(h, SWEPT_EINVAL, "ckpt_dev NULL or not 256-byte aligned, or nsteps < 0");
  const int64_t K = adj_segment(h, nsteps, bytes);
  if (nsteps > 0 && K <= 0) return fail(h, SWEPT_ENOMEM_WORKSPACE, "ckpt_bytes too small for one pass per segment");
  *plan = adj_layout(h, nsteps, nsteps > 0 ? K : 1);
  if (plan->bytes > bytes) return fail(h, SWEPT_ENOMEM_WORKSPACE, "ckpt_bytes too small");
  return SWEPT_OK;
}

swept_status forward_ckpt(swept_handle* h, void* u, int64_t nsteps, char* ck, size_t bytes, const AdjPlan& a,
                          cudaStream_t s) {
  const int64_t NC = h->g.N * h->g.C;
  const size_t slot = align_up((size_t)NC * sizeof(double));
  for (int64_t sg = 0; sg < a.nseg; ++sg) {
    const int64_t Ks = std::min(a.K, nsteps - sg * a.K);
    cudaError_t e = h->impl->copy(NC, u, ck + a.off_ck + (size_t)sg * slot, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint copy");
    if (sg + 1 < a.nseg) {
      swept_status st = swept_step_n(h, u, Ks, s);
      if (st != SWEPT_OK) return st;
    } else {
      e = h->impl->copy(NC, u, ck + a.off_tape, s);
      if (e == cudaSuccess) e = issue_swept_tape(h, u, Ks * h->g.S, ck + a.off_tape, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "tape-recording forward");
    }
  }
  h->fwd_ckpt = ck;
  h->fwd_nsteps = nsteps;
  h->fwd_bytes = bytes;
  h->fwd_tape_valid = true;
  return SWEPT_OK;
}

}  // namespace

extern "C" {

swept_status swept_init(const swept_config* cfg, swept_handle** out) {
  if (!cfg || !out) return SWEPT_EINVAL;
  *out = nullptr;
  const SchemeImpl* im = pick_impl(cfg->scheme, cfg->dtype);
  if (!im) return SWEPT_EINVAL;
  if (cfg->bc != SWEPT_BC_PERIODIC && cfg->bc != SWEPT_BC_REFLECTIVE) return SWEPT_EINVAL;
  if (cfg->scheme == SWEPT_KS && cfg->bc != SWEPT_BC_PERIODIC) return SWEPT_EINVAL;
  if (!(cfg->dx > 0) || !(cfg->dt > 0) || cfg->n < 2 * im->R + 1) return SWEPT_EINVAL;
  if (cfg->scheme == SWEPT_EULER && !(cfg->param[0] > 1.0)) return SWEPT_EINVAL;
  swept_handle* h = new (std::nothrow) swept_handle();
  if (!h) return SWEPT_EINVAL;
  h->cfg = *cfg;
  h->impl = im;
  // Plan from the current device's properties; without a usable device the
  // plan uses GB300's (152 SMs, 227 KB opt-in shared memory) so that the host
  // schedule check still works, and every compute call fails with SWEPT_ECUDA.
  int max_smem = kGb300SmemOptin;
  h->sm_count = kGb300Sms;
  h->device = -1;
  int dev = -1;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int sms = 0, sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) {
      h->device = dev;
      h->sm_count = sms;
      max_smem = sm;
    }
  }
  cudaGetLastError();  // clear a no-device error
  cudaError_t e = cudaSuccess;
  const int R = im->R;
  const int W = cfg->tile_w > 0 ? cfg->tile_w : choose_tile(cfg->n, R, h->sm_count);
  // an explicit tile must be legal; with the library's choice, a grid too
  // small for two tiles of 4R points still gets a handle for classic_step_n
  if (cfg->tile_w != 0 && (cfg->tile_w < 0 || !tile_ok(cfg->n, W, R))) {
    delete h;
    return SWEPT_EINVAL;
  }
  h->tiled = W > 0;
  Geom& g = h->g;
  g.N = cfg->n;
  g.R = R;
  g.S = im->S;
  g.C = im->C;
  g.bc = cfg->bc;
  if (h->tiled) {
    g.W = W;
    g.h = W / (2 * R);
    g.nt = cfg->n / W;
    g.X = (int)(cfg->n - g.nt * W);
    g.M = (W + g.X + 2 * R + 1) / 2 * 2;  // even row stride: paired (8- / 16-byte) loads stay aligned
    g.E = 2 * g.h * g.C * 2 * R;
  }
  // one point per thread per tier unless asked: on GB300 the register-window
  // mapping measured slower at every size (the tiers are latency-bound, and
  // spreading a tier over more warps beats fewer shared-memory reads)
  g.chunk = cfg->chunk > 0 ? cfg->chunk : 1;
  if (g.chunk != 1 && g.chunk != 2) {  // heat/KS: strided pairs; Euler: two threads per face
    delete h;
    return SWEPT_EINVAL;
  }
  int th = cfg->threads > 0 ? cfg->threads : (W >= 256 ? 256 : std::max(32, ((W + 31) / 32) * 32));
  if (th < 32 || th > 1024 || th % 32 != 0) {
    delete h;
    return SWEPT_EINVAL;
  }
  // tiers in registers: one warp per tile, W / 32 points per lane
  if (cfg->warp_tiles != 0 && cfg->warp_tiles != 1) {
    delete h;
    return SWEPT_EINVAL;
  }
  if (cfg->warp_tiles == 1) {
    const int P = W / 32;
    if (!h->tiled || g.X != 0 || im->C != 1 || W % 32 != 0 || (P != 1 && P != 2 && P != 4 && P != 8) ||
        g.chunk != 1 || (cfg->threads != 0 && cfg->threads != 32)) {
      delete h;
      return SWEPT_EINVAL;
    }
    g.P = P;
    th = 32;
  }
  h->threads = th;
  h->smem = h->tiled ? (size_t)im->smem_values(g.M) * im->value_bytes : 0;
  if (h->smem > (size_t)max_smem) {
    delete h;
    return SWEPT_EINVAL;
  }
  im->make_consts(cfg->param, cfg->dx, cfg->dt, h->k);
  const size_t vb = (size_t)im->value_bytes;
  const size_t ebytes = align_up((size_t)swept::edge_slots(g) * g.E * vb);
  h->off_e0 = 0;
  h->off_e1 = ebytes;
  h->off_tmp = 2 * ebytes;
  h->off_status = h->off_tmp + align_up((size_t)g.N * g.C * vb);
  h->off_persist = h->off_status + kAlign;
  h->ws_bytes = h->off_persist + align_up((size_t)g.nt * sizeof(int)) + kAlign;
  if (cfg->persistent != 0 && cfg->persistent != 1) {
    delete h;
    return SWEPT_EINVAL;
  }
  h->persistent = cfg->persistent == 1;
  if (cfg->cluster != 0 && cfg->cluster != 1) {
    delete h;
    return SWEPT_EINVAL;
  }
  h->cluster = cfg->cluster == 1;
  if ((h->persistent || h->cluster) && !h->tiled) {
    delete h;
    return SWEPT_EINVAL;
  }
  if (h->cluster && (g.nt > 16 || g.X != 0 || h->persistent ||
                     h->smem + 2 * (size_t)g.E * im->value_bytes > (size_t)max_smem)) {
    delete h;
    return SWEPT_EINVAL;
  }
  (void)e;
  *out = h;
  return SWEPT_OK;
}

swept_status swept_workspace_size(const swept_handle* h, size_t* bytes) {
  if (!h || !bytes) return SWEPT_EINVAL;
  *bytes = h->ws_bytes;
  return SWEPT_OK;
}

swept_status swept_bind_workspace(swept_handle* h, void* ws_dev, size_t bytes) {
  if (!h) return SWEPT_EINVAL;
  if (!ws_dev || ((uintptr_t)ws_dev % kAlign) != 0) return fail(h, SWEPT_EINVAL, "workspace NULL or not 256-byte aligned");
  if (bytes < h->ws_bytes) return fail(h, SWEPT_ENOMEM_WORKSPACE, "workspace smaller than swept_workspace_size()");
  swept_status st = ensure_device(h);
  if (st != SWEPT_OK) return st;
  drop_graphs(h);
  h->ws = (char*)ws_dev;
  h->ws_bound = bytes;
  cudaError_t e = cudaMemset(h->ws + h->off_status, 0, kAlign);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset(status)");
  return SWEPT_OK;
}

swept_status swept_step_n(swept_handle* h, void* u_dev, int64_t nsteps, void* stream) {
  const swept_trace::Range trace_range("swept_step_n");
  swept_status st = check_ready(h, u_dev, nsteps);
  if (st != SWEPT_OK) return st;
  if (!h->tiled) return no_tiling(h);
  if (nsteps == 0) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t n_sub = nsteps * h->g.S;
  if (h->cluster) {
    return run_graph(h, key_of("swept_cluster", u_dev, nsteps), s, [&](cudaStream_t cs) {
      return h->impl->cluster(h->g, h->k, u_dev, n_sub, h->threads, h->smem, cs);
    });
  }
  if (h->persistent) {
    if (!h->persist_blocks) {
      const int per_sm = h->impl->persist_blocks_per_sm(h->g.P, h->threads, h->smem);
      if (per_sm < 1) return fail(h, SWEPT_EINVAL, "persistent kernel does not fit on an SM");
      h->persist_blocks = per_sm * h->sm_count;
    }
    const Geom& g = h->g;
    const int64_t q = n_sub / g.h, rem = n_sub % g.h;
    const int64_t items = ((q > 0 ? q + 1 : 0) + (rem > 0 ? 2 : 0)) * g.nt;
    const int blocks = (int)std::min<int64_t>(items, h->persist_blocks);
    char* pc = h->ws + h->off_persist;
    int* done = (int*)pc;
    char* ctl = pc + align_up((size_t)g.nt * sizeof(int));
    return run_graph(h, key_of("swept_persist", u_dev, nsteps), s, [&](cudaStream_t cs) {
      cudaError_t e = cudaMemsetAsync(pc, 0xFF, (size_t)g.nt * sizeof(int), cs);
      if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, 16, cs);
      if (e == cudaSuccess)
        e = h->impl->persist(g, h->k, u_dev, h->ws + h->off_e0, h->ws + h->off_e1, n_sub, done,
                             (unsigned long long*)ctl, (int*)(ctl + 8), h->spin_limit, h->start_item, blocks,
                             h->threads, h->smem, cs);
      // a wait that ran out is latched into the handle's status word
      if (e == cudaSuccess) {
        swept::k_latch_error<<<1, 1, 0, cs>>>((const int*)(ctl + 8), (int*)(h->ws + h->off_status));
        e = cudaGetLastError();
      }
      return e;
    });
  }
  const int64_t L = swept_launch_count(h->g, n_sub);
  const int64_t kChunk = 512;  // diamond passes per cached body graph
  if (L <= 2 * kChunk + 4) {
    return run_graph(h, key_of("swept", u_dev, nsteps), s,
                     [&](cudaStream_t cs) { return issue_swept(h, u_dev, n_sub, 0, L, cs); });
  }
  // head (up-triangle), a reusable body of kChunk diamonds (even count, so
  // pass parities and edge buffers repeat), then the tail
  const int64_t q = n_sub / h->g.h;
  const int64_t reps = (q - 1) / kChunk;
  st = run_graph(h, key_of("swept_head", u_dev, 0), s,
                 [&](cudaStream_t cs) { return issue_swept(h, u_dev, n_sub, 0, 1, cs); });
  if (st != SWEPT_OK) return st;
  for (int64_t r = 0; r < reps; ++r) {
    st = run_graph(h, key_of("swept_body", nullptr, kChunk), s,
                   [&](cudaStream_t cs) { return issue_swept(h, u_dev, n_sub, 1, 1 + kChunk, cs); });
    if (st != SWEPT_OK) return st;
  }
  const int64_t t0 = 1 + reps * kChunk;
  return run_graph(h, key_of("swept_tail", u_dev, nsteps), s,
                   [&](cudaStream_t cs) { return issue_swept(h, u_dev, n_sub, t0, L, cs); });
}

swept_status classic_step_n(swept_handle* h, void* u_dev, int64_t nsteps, void* stream) {
  const swept_trace::Range trace_range("classic_step_n");
  swept_status st = check_ready(h, u_dev, nsteps);
  if (st != SWEPT_OK || nsteps == 0) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t S = h->g.S;
  const int64_t n_sub = nsteps * S;
  const int64_t kBody = 512;  // full steps per cached body graph (even: heat returns to u)
  const int64_t reps = nsteps / kBody;
  for (int64_t r = 0; r < reps; ++r) {
    st = run_graph(h, key_of("classic_body", u_dev, kBody), s,
                   [&](cudaStream_t cs) { return issue_classic(h, u_dev, 0, kBody * S, cs); });
    if (st != SWEPT_OK) return st;
  }
  const int64_t k0 = reps * kBody * S;
  if (k0 == n_sub) return SWEPT_OK;
  return run_graph(h, key_of("classic_tail", u_dev, nsteps - reps * kBody), s, [&](cudaStream_t cs) {
    cudaError_t e = issue_classic(h, u_dev, k0, n_sub, cs);
    if (e == cudaSuccess && S == 1 && (n_sub & 1))
      e = h->impl->copy(h->g.N * h->g.C, h->ws + h->off_tmp, u_dev, cs);
    return e;
  });
}

swept_status swept_run_host(swept_handle* h, const void* u_host_in, void* u_host_out, void* u_dev, int64_t nsteps,
                            int32_t use_swept, void* stream) {
  const swept_trace::Range trace_range("swept_run_host");
  if (!h) return SWEPT_EINVAL;
  if (!u_host_in || !u_host_out) return fail(h, SWEPT_EINVAL, "host buffer is NULL");
  if (use_swept && !h->tiled) return no_tiling(h);
  swept_status st = check_ready(h, u_dev, nsteps);
  if (st != SWEPT_OK) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)h->g.N * h->g.C * h->impl->value_bytes;
  cudaError_t e = cudaMemcpyAsync(u_dev, u_host_in, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync H2D");
  st = use_swept ? swept_step_n(h, u_dev, nsteps, stream) : classic_step_n(h, u_dev, nsteps, stream);
  if (st != SWEPT_OK) return st;
  e = cudaMemcpyAsync(u_host_out, u_dev, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync D2H");
  e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SWEPT_OK : cuda_fail(h, e, "cudaStreamSynchronize");
}

swept_status swept_adjoint_ckpt_size(const swept_handle* h, int64_t nsteps, size_t* bytes) {
  if (!h || !bytes || nsteps < 0) return SWEPT_EINVAL;
  if (!h->impl->adj_up || h->cfg.dtype != SWEPT_F64 || !h->tiled) return SWEPT_EUNSUPPORTED;
  *bytes = adj_layout(h, nsteps, std::max<int64_t>(1, adj_segment(h, nsteps, 0))).bytes;
  return SWEPT_OK;
}

swept_status swept_forward_ckpt(swept_handle* h, void* u_dev, int64_t nsteps, void* ckpt_dev, size_t ckpt_bytes,
                                void* stream) {
  const swept_trace::Range trace_range("swept_forward_ckpt");
  swept_status st = check_ready(h, u_dev, nsteps);
  if (st != SWEPT_OK) return st;
  AdjPlan a;
  st = adj_check(h, nsteps, ckpt_dev, ckpt_bytes, &a);
  if (st != SWEPT_OK || nsteps == 0) return st;
  return forward_ckpt(h, u_dev, nsteps, (char*)ckpt_dev, ckpt_bytes, a, (cudaStream_t)stream);
}

swept_status swept_adjoint(swept_handle* h, const void* u0_dev, const void* gT_dev, int64_t nsteps, void* g_u0_dev,
                           void* g_param_dev, void* ckpt_dev, size_t ckpt_bytes, void* stream) {
  const swept_trace::Range trace_range("swept_adjoint");
  swept_status st = check_ready(h, g_u0_dev, nsteps);
  if (st != SWEPT_OK) return st;
  if (!gT_dev || !g_param_dev) return fail(h, SWEPT_EINVAL, "gT_dev or g_param_dev is NULL");
  AdjPlan a;
  st = adj_check(h, nsteps, ckpt_dev, ckpt_bytes, &a);
  if (st != SWEPT_OK) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  char* ck = (char*)ckpt_dev;
  const int64_t NC = h->g.N * h->g.C;
  const size_t slot = align_up((size_t)NC * sizeof(double));
  void* lam = ck + a.off_lam;
  void* w = ck + a.off_w;
  double* slots = (double*)(ck + a.off_slots);
  cudaError_t e;
  if (u0_dev) {
    e = h->impl->copy(NC, u0_dev, w, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy u0");
    if (nsteps > 0) {
      st = forward_ckpt(h, w, nsteps, ck, ckpt_bytes, a, s);
      if (st != SWEPT_OK) return st;
    }
  } else if (nsteps > 0 && !(h->fwd_ckpt == ckpt_dev && h->fwd_nsteps == nsteps && h->fwd_bytes == ckpt_bytes)) {
    return fail(h, SWEPT_EINVAL, "u0_dev is NULL but no swept_forward_ckpt with this ckpt_dev/nsteps/ckpt_bytes");
  }
  unsigned char ka[swept::KBYTES];
  h->impl->make_adj_consts(h->cfg.param, h->cfg.dx, h->cfg.dt, ka);
  const size_t sm = adj_smem(h);
  if (sm > 48 * 1024) {
    e = h->impl->adj_prepare(sm);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint shared-memory limit");
  }
  e = cudaMemsetAsync(slots, 0, (size_t)2 * h->g.nt * sizeof(double), s);
  if (e == cudaSuccess) e = h->impl->copy(NC, gT_dev, lam, s);
  for (int64_t sg = a.nseg - 1; sg >= 0 && e == cudaSuccess && nsteps > 0; --sg) {
    const int64_t Ks = std::min(a.K, nsteps - sg * a.K);
    if (!(sg == a.nseg - 1 && h->fwd_tape_valid)) {
      e = h->impl->copy(NC, ck + a.off_ck + (size_t)sg * slot, ck + a.off_tape, s);
      if (e == cudaSuccess) e = h->impl->copy(NC, ck + a.off_ck + (size_t)sg * slot, w, s);
      if (e == cudaSuccess) e = issue_swept_tape(h, w, Ks * h->g.S, ck + a.off_tape, s);
    }
    if (e == cudaSuccess) e = issue_adjoint(h, ka, lam, Ks * h->g.S, ck + a.off_tape, slots, s);
  }
  if (a.nseg > 1) h->fwd_tape_valid = false;  // the tape now holds the first segment
  if (e == cudaSuccess) e = h->impl->copy(NC, lam, g_u0_dev, s);
  if (e == cudaSuccess) {
    swept::k_sum_slots<<<1, 32, 0, s>>>(slots, h->g.nt, (double*)g_param_dev);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? SWEPT_OK : cuda_fail(h, e, "swept_adjoint");
}

swept_status swept_profile_passes(swept_handle* h, void* u_dev, int64_t nsteps, void* stream, double* out_ms,
                                  int64_t* out_count) {
  swept_status st = check_ready(h, u_dev, nsteps);
  if (st != SWEPT_OK) return st;
  if (!h->tiled) return no_tiling(h);
  if (!out_ms || !out_count) return fail(h, SWEPT_EINVAL, "NULL output arrays");
  for (int i = 0; i < 4; ++i) {
    out_ms[i] = 0.0;
    out_count[i] = 0;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t n_sub = nsteps * h->g.S;
  const int64_t L = swept_launch_count(h->g, n_sub);
  std::vector<cudaEvent_t> ev((size_t)(2 * L), nullptr);
  std::vector<int> kind((size_t)L, 0);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  int64_t idx = 0;
  if (e == cudaSuccess) {
    swept::for_each_launch(h->g, n_sub, [&](int k, int, int mode, int, int64_t pass) {
      kind[(size_t)idx] = pass < 0 ? 3 : (k == 0 ? 0 : (mode == swept::MODE_DOWN ? 2 : 1));
      ++idx;
    });
    for (int64_t i = 0; i < L && e == cudaSuccess; ++i) {
      e = cudaEventRecord(ev[(size_t)(2 * i)], s);
      if (e == cudaSuccess) e = issue_swept(h, u_dev, n_sub, i, i + 1, s);
      if (e == cudaSuccess) e = cudaEventRecord(ev[(size_t)(2 * i + 1)], s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int64_t i = 0; i < L && e == cudaSuccess; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[(size_t)(2 * i)], ev[(size_t)(2 * i + 1)]);
      out_ms[kind[(size_t)i]] += ms;
      out_count[kind[(size_t)i]] += 1;
    }
  }
  for (auto x : ev)
    if (x) cudaEventDestroy(x);
  return e == cudaSuccess ? SWEPT_OK : cuda_fail(h, e, "swept_profile_passes");
}

swept_status swept_get_plan(const swept_handle* h, swept_plan_info* out) {
  if (!h || !out) return SWEPT_EINVAL;
  out->tile_w = h->g.W;
  out->threads = h->threads;
  out->half_cycle = h->g.h;
  out->radius = h->g.R;
  out->stages = h->g.S;
  out->components = h->g.C;
  out->tiles = h->g.nt;
  out->smem_bytes = (int64_t)h->smem;
  out->workspace_bytes = (int64_t)h->ws_bytes;
  out->chunk = h->g.chunk;
  out->persistent = h->persistent ? 1 : 0;
  out->cluster = h->cluster ? 1 : 0;
  out->warp_tiles = h->g.P > 0 ? 1 : 0;
  out->last_tile_extra = h->g.X;
  return SWEPT_OK;
}

swept_status swept_sync_status(swept_handle* h, void* stream) {
  if (!h) return SWEPT_EINVAL;
  if (!h->ws) return fail(h, SWEPT_ENOWORKSPACE, "no workspace bound");
  const cudaStream_t s = (cudaStream_t)stream;
  int32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, h->ws + h->off_status, sizeof word, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->off_status, 0, sizeof word, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "swept_sync_status");
  if (word == 0) return SWEPT_OK;
  return fail(h, word == SWEPT_ETIMEOUT ? SWEPT_ETIMEOUT : SWEPT_EDEVICE, "device-side error word set");
}

}  // extern "C"

namespace swept {

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, fn);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

namespace dbg {
namespace {
std::vector<FetchFn>& fetchers() {
  static std::vector<FetchFn> v;
  return v;
}
__global__ void k_debug_probe(double* buf, int64_t n, int64_t bound) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (in_range(i, bound, PROBE)) buf[i] = buf[i];
}
}  // namespace
void register_fetch(FetchFn f) { fetchers().push_back(f); }
}  // namespace dbg
}  // namespace swept

extern "C" {

swept_status swept_debug_status(int32_t* enabled, int32_t* check, int64_t* index) {
  if (enabled) *enabled = SWEPT_DEBUG;
  if (check) *check = 0;
  if (index) *index = 0;
  if (!SWEPT_DEBUG) return SWEPT_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) return SWEPT_ECUDA;
  unsigned long long first = 0;
  for (swept::dbg::FetchFn f : swept::dbg::fetchers()) {
    unsigned long long w = 0;
    if (f(&w) != cudaSuccess) return SWEPT_ECUDA;
    if (!first) first = w;
  }
  if (!first) return SWEPT_OK;
  if (check) *check = (int32_t)(first >> 48);
  if (index) {
    int64_t v = (int64_t)(first & 0xffffffffffffULL);
    if (v & (1LL << 47)) v -= (1LL << 48);  // sign of the 48-bit field
    *index = v;
  }
  return SWEPT_EDEVICE;
}

swept_status swept_debug_probe(double* buf, int64_t n, int64_t bound, void* stream) {
  if (n < 0 || bound < 0 || bound > n || (n > 0 && !buf)) return SWEPT_EINVAL;
  if (n == 0) return SWEPT_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
  swept::dbg::k_debug_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(buf, n, bound);
  return cudaGetLastError() == cudaSuccess ? SWEPT_OK : SWEPT_ECUDA;
}

swept_status swept_set_option(swept_handle* h, int32_t option, int64_t value) {
  if (!h) return SWEPT_EINVAL;
  if (option == SWEPT_OPT_SPIN_LIMIT) {
    if (value < 1 || value > 0xffffffffLL) return fail(h, SWEPT_EINVAL, "spin limit outside [1, 2^32)");
    h->spin_limit = (uint32_t)value;
  } else if (option == SWEPT_OPT_START_ITEM) {
    if (value < 0) return fail(h, SWEPT_EINVAL, "start item < 0");
    h->start_item = value;
  } else {
    return fail(h, SWEPT_EINVAL, "unknown option");
  }
  drop_graphs(h);  // captured persistent launches carry the options
  return SWEPT_OK;
}

swept_status swept_check_schedule(swept_handle* h, int64_t nsteps, int64_t* computed_out) {
  if (!h || nsteps < 0) return SWEPT_EINVAL;
  if (!h->tiled) return no_tiling(h);
  return swept::check_schedule(h, nsteps, computed_out);
}

swept_status swept_last_error(const swept_handle* h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return SWEPT_EINVAL;
  snprintf(buf, len, "%s", h->err.c_str());
  return SWEPT_OK;
}

void swept_free(swept_handle* h) {
  if (!h) return;
  drop_graphs(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

}  // extern "C"
