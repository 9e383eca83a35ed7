// C-ABI runtime of the 2D swept solver (include/swept2d.h): plan, workspace
// layout, launch sequence of the swept path (per pass, or the persistent queue
// kernel) and of the classic path, CUDA-graph caching.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <new>
#include <string>

#include "graph_cache.h"
#include "impl.h"
#include "kernels2d.cuh"
#include "swept2d.h"
#include "trace.h"

using swept2d::Geom2;

struct swept2d_handle {
  swept2d_config cfg;
  Geom2 g;
  int threads = 256;
  size_t smem = 0;
  int device = -1;
  int value_bytes = 8;
  double fo = 0.0;  // alpha dt / dx^2, in double
  bool persistent = false;
  int persist_blocks = 0;  // resident blocks of the persistent kernel (0: not yet known)
  int sm_count = 0;
  uint32_t spin_limit = 1u << 24;
  int64_t start_item = 0;
  int64_t check_drop_wait = -1;  // replay only: an item whose last wait is dropped
  char* ws = nullptr;
  size_t ws_bytes = 0, ws_bound = 0;
  size_t off_s0 = 0, off_s1 = 0, off_b = 0, off_b1 = 0, off_tmp = 0, off_status = 0, off_persist = 0;
  cudaStream_t cap = nullptr;
  std::map<std::string, cudaGraphExec_t> graphs;
  std::string err;
};

namespace swept2d {
// symbolic replay of the 2D launch sequence or persistent queue (check2d.cpp)
bool check_schedule2d(const Geom2& g, int64_t nsteps, bool persistent, int64_t drop_wait, int64_t* computed,
                      std::string* err);
}  // namespace swept2d

namespace {

constexpr size_t kAlign = 256;
constexpr int kSmemOptin = 232448;  // GB300 opt-in shared memory per block
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

swept_status fail(swept2d_handle* h, swept_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}
swept_status cuda_fail(swept2d_handle* h, cudaError_t e, const char* where) {
  return fail(h, SWEPT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int max_tile(int dtype) { return dtype == SWEPT_F64 ? 64 : 128; }
bool tile_ok(int64_t nx, int64_t ny, int W, int dtype) {
  return W >= 8 && W <= max_tile(dtype) && W % 4 == 0 && nx % W == 0 && ny % W == 0 && nx / W >= 2 && ny / W >= 2;
}
// default: 32 where it fits (the measured best at 2^20 points), else the largest legal W
int choose_tile(int64_t nx, int64_t ny, int dtype) {
  if (tile_ok(nx, ny, 32, dtype)) return 32;
  for (int W = max_tile(dtype); W >= 8; W -= 4)
    if (tile_ok(nx, ny, W, dtype)) return W;
  return 0;
}


swept_status run_graph(swept2d_handle* h, const std::string& key, cudaStream_t user,
                       const std::function<cudaError_t(cudaStream_t)>& issue) {
  return swept_graphs::run(h, key, user, issue);
}
void drop_graphs(swept2d_handle* h) { swept_graphs::drop(h); }
using swept_graphs::key_of;

template <typename T>
cudaError_t prepare_t(size_t smem) {
  cudaError_t e = swept::raise_smem_limit((const void*)swept2d::k_pyr2d<T>, smem);
  if (e == cudaSuccess) e = swept::raise_smem_limit((const void*)swept2d::k_bridge2d<T>, smem);
  if (e == cudaSuccess) e = swept::raise_smem_limit((const void*)swept2d::k_octa2d<T>, smem);
  if (e == cudaSuccess) e = swept::raise_smem_limit((const void*)swept2d::k_persist2d<T>, smem);
  return e;
}

swept_status ensure_device(swept2d_handle* h) {
  if (h->device < 0) return fail(h, SWEPT_ECUDA, "no CUDA device was available when the handle was created");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
  if (dev != h->device) return fail(h, SWEPT_EINVAL, "current device differs from the handle's device");
  if (!h->cap) {
    if (h->smem > 48 * 1024) {
      e = h->value_bytes == 8 ? prepare_t<double>(h->smem) : prepare_t<float>(h->smem);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
    }
    e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreateWithFlags");
  }
  return SWEPT_OK;
}

swept_status check_ready(swept2d_handle* h, void* u_dev, int64_t nsteps) {
  if (!h) return SWEPT_EINVAL;
  if (!u_dev || nsteps < 0) return fail(h, SWEPT_EINVAL, "u_dev is NULL or nsteps < 0");
  if (!h->ws) return fail(h, SWEPT_ENOWORKSPACE, "no workspace bound (swept2d_bind_workspace)");
  if (h->ws_bound < h->ws_bytes) return fail(h, SWEPT_ENOMEM_WORKSPACE, "bound workspace too small");
  return ensure_device(h);
}

template <typename T>
swept2d::Heat2dK<T> consts(const swept2d_handle* h) {
  swept2d::Heat2dK<T> k;
  k.fo = (T)h->fo;
  k.c1 = (T)(1.0 - 4.0 * h->fo);
  return k;
}

// launches [from, to) of for_each_launch2d
template <typename T>
cudaError_t issue_swept_t(swept2d_handle* h, T* u, int64_t n, int64_t from, int64_t to, cudaStream_t s) {
  const Geom2& g = h->g;
  const auto k = consts<T>(h);
  T* S[2] = {(T*)(h->ws + h->off_s0), (T*)(h->ws + h->off_s1)};
  T* B = (T*)(h->ws + h->off_b);
  const unsigned tiles = (unsigned)(g.ntx * g.nty);
  int64_t idx = 0;
  cudaError_t err = cudaSuccess;
  swept2d::for_each_launch2d(g, n, [&](int kind, int par, int mode, int hh, int64_t c) {
    const int64_t i = idx++;
    if (err != cudaSuccess || i < from || i >= to) return;
    const int in = c >= 1 ? (int)((c - 1) & 1) : 0;
    const int out = c >= 0 ? (int)(c & 1) : 1;
    if (kind == swept2d::K_PYR)
      swept2d::k_pyr2d<T><<<tiles, h->threads, h->smem, s>>>(g, k, u, S[c >= 0 ? out : 0], par, hh,
                                                              mode == swept2d::M2_GAP);
    else if (kind == swept2d::K_BRIDGE)
      swept2d::k_bridge2d<T><<<2 * tiles, h->threads, h->smem, s>>>(g, k, u, S[in], B, par, hh,
                                                                     mode == swept2d::M2_GAP);
    else
      swept2d::k_octa2d<T><<<tiles, h->threads, h->smem, s>>>(g, k, u, S[in], S[out], B, par, mode, hh);
    err = cudaGetLastError();
  });
  return err;
}

// the persistent form: counters reset, one launch over the whole queue, the
// error word latched into the status word
template <typename T>
cudaError_t issue_persist_t(swept2d_handle* h, T* u, int64_t n, cudaStream_t s) {
  const Geom2& g = h->g;
  const size_t T_ = (size_t)(g.ntx * g.nty);
  char* pc = h->ws + h->off_persist;
  int* tile_done = (int*)pc;
  int* bridge_done = tile_done + T_;
  char* ctl = pc + align_up(3 * T_ * sizeof(int));
  cudaError_t e = cudaMemsetAsync(pc, 0xFF, 3 * T_ * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, 16, s);
  if (e != cudaSuccess) return e;
  swept2d::Persist2Ctl c{tile_done, bridge_done, (unsigned long long*)ctl, (int*)(ctl + 8), h->spin_limit,
                         h->start_item};
  const int64_t items = swept2d::persist2d_items(g, n);
  const unsigned blocks = (unsigned)std::min<int64_t>(items, h->persist_blocks);
  swept2d::k_persist2d<T><<<blocks, h->threads, h->smem, s>>>(
      g, consts<T>(h), u, (T*)(h->ws + h->off_s0), (T*)(h->ws + h->off_s1), (T*)(h->ws + h->off_b),
      (T*)(h->ws + h->off_b1), n, c);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    swept2d::k_latch_error2d<<<1, 1, 0, s>>>((const int*)(ctl + 8), (int*)(h->ws + h->off_status));
    e = cudaGetLastError();
  }
  return e;
}

template <typename T>
int persist_blocks_per_sm_t(const swept2d_handle* h) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, swept2d::k_persist2d<T>, h->threads, h->smem) != cudaSuccess)
    return 0;
  return n;
}

cudaError_t issue_swept(swept2d_handle* h, void* u, int64_t n, int64_t from, int64_t to, cudaStream_t s) {
  return h->value_bytes == 8 ? issue_swept_t<double>(h, (double*)u, n, from, to, s)
                             : issue_swept_t<float>(h, (float*)u, n, from, to, s);
}

// classic steps [k0, k1): step m reads u (m even) or the second array and
// writes the other; an odd total leaves the result in u by a final copy
template <typename T>
cudaError_t issue_classic_t(swept2d_handle* h, T* u, int64_t k0, int64_t k1, int64_t total, cudaStream_t s) {
  const Geom2& g = h->g;
  const auto k = consts<T>(h);
  T* tmp = (T*)(h->ws + h->off_tmp);
  const dim3 grid((unsigned)((g.nx + 255) / 256), (unsigned)g.ny);
  for (int64_t m = k0; m < k1; ++m) {
    const T* in = (m & 1) ? tmp : u;
    T* out = (m & 1) ? u : tmp;
    swept2d::k_classic2d<T><<<grid, 256, 0, s>>>(g.nx, g.ny, g.bc, k, in, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (k1 == total && (total & 1))
    return cudaMemcpyAsync(u, tmp, (size_t)(g.nx * g.ny) * sizeof(T), cudaMemcpyDeviceToDevice, s);
  return cudaSuccess;
}

cudaError_t issue_classic(swept2d_handle* h, void* u, int64_t k0, int64_t k1, int64_t total, cudaStream_t s) {
  return h->value_bytes == 8 ? issue_classic_t<double>(h, (double*)u, k0, k1, total, s)
                             : issue_classic_t<float>(h, (float*)u, k0, k1, total, s);
}

}  // namespace

extern "C" {

swept_status swept2d_init(const swept2d_config* cfg, swept2d_handle** out) {
  if (!cfg || !out) return SWEPT_EINVAL;
  *out = nullptr;
  if (cfg->dtype != SWEPT_F32 && cfg->dtype != SWEPT_F64) return SWEPT_EINVAL;
  if (cfg->bc != SWEPT_BC_PERIODIC && cfg->bc != SWEPT_BC_REFLECTIVE) return SWEPT_EINVAL;
  if (!(cfg->dx > 0) || !(cfg->dt > 0) || !(cfg->alpha > 0)) return SWEPT_EINVAL;
  if (cfg->nx < 16 || cfg->ny < 16 || cfg->ny > 65535) return SWEPT_EINVAL;
  const int W = cfg->tile_w > 0 ? cfg->tile_w : choose_tile(cfg->nx, cfg->ny, cfg->dtype);
  if (W <= 0 || !tile_ok(cfg->nx, cfg->ny, W, cfg->dtype)) return SWEPT_EINVAL;
  const int th = cfg->threads > 0 ? cfg->threads : 256;
  if (th < 32 || th > 1024 || th % 32 != 0) return SWEPT_EINVAL;
  if (cfg->persistent != 0 && cfg->persistent != 1) return SWEPT_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (cfg->reserved[i] != 0) return SWEPT_EINVAL;
  swept2d_handle* h = new (std::nothrow) swept2d_handle();
  if (!h) return SWEPT_EINVAL;
  h->cfg = *cfg;
  h->threads = th;
  h->persistent = cfg->persistent == 1;
  h->value_bytes = cfg->dtype == SWEPT_F64 ? 8 : 4;
  h->fo = cfg->alpha * cfg->dt / (cfg->dx * cfg->dx);
  Geom2& g = h->g;
  g.nx = cfg->nx;
  g.ny = cfg->ny;
  g.W = W;
  g.R = 1;
  g.h = W / 2;
  g.M = W + 2;
  g.ntx = cfg->nx / W;
  g.nty = cfg->ny / W;
  g.Ph = swept2d::strip_off(g, g.h);
  g.Bh = swept2d::band_off(g, g.h);
  g.Es = 4 * 2 * g.R * g.Ph;
  g.Eb = 2 * 2 * g.R * g.Bh;
  g.bc = cfg->bc;
  h->smem = (size_t)2 * g.M * g.M * h->value_bytes;
  if (h->smem > (size_t)kSmemOptin) {
    delete h;
    return SWEPT_EINVAL;
  }
  const size_t vb = (size_t)h->value_bytes;
  const size_t strips = align_up((size_t)(g.ntx * g.nty * g.Es) * vb);
  const size_t bands = align_up((size_t)(2 * g.ntx * g.nty * g.Eb) * vb);
  h->off_s0 = 0;
  h->off_s1 = strips;
  h->off_b = 2 * strips;
  // the persistent kernel overlaps half cycles, so it double-buffers the bands too
  h->off_b1 = h->off_b + bands;
  h->off_tmp = h->off_b1 + (h->persistent ? bands : 0);
  h->off_status = h->off_tmp + align_up((size_t)(g.nx * g.ny) * vb);
  h->off_persist = h->off_status + kAlign;
  const size_t T_ = (size_t)(g.ntx * g.nty);
  h->ws_bytes = h->off_persist + (h->persistent ? align_up(3 * T_ * sizeof(int)) + kAlign : 0);
  int dev = -1;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int n = 0;
    if (cudaGetDeviceCount(&n) == cudaSuccess && n > 0) {
      h->device = dev;
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
  }
  cudaGetLastError();  // clear a no-device error
  *out = h;
  return SWEPT_OK;
}

swept_status swept2d_workspace_size(const swept2d_handle* h, size_t* bytes) {
  if (!h || !bytes) return SWEPT_EINVAL;
  *bytes = h->ws_bytes;
  return SWEPT_OK;
}

swept_status swept2d_bind_workspace(swept2d_handle* h, void* ws_dev, size_t bytes) {
  if (!h) return SWEPT_EINVAL;
  if (!ws_dev || ((uintptr_t)ws_dev % kAlign) != 0)
    return fail(h, SWEPT_EINVAL, "workspace NULL or not 256-byte aligned");
  if (bytes < h->ws_bytes) return fail(h, SWEPT_ENOMEM_WORKSPACE, "workspace smaller than swept2d_workspace_size()");
  swept_status st = ensure_device(h);
  if (st != SWEPT_OK) return st;
  drop_graphs(h);
  h->ws = (char*)ws_dev;
  h->ws_bound = bytes;
  cudaError_t e = cudaMemset(h->ws + h->off_status, 0, kAlign);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset(status)");
  return SWEPT_OK;
}

swept_status swept2d_step_n(swept2d_handle* h, void* u_dev, int64_t nsteps, void* stream) {
  const swept_trace::Range trace_range("swept2d_step_n");
  swept_status st = check_ready(h, u_dev, nsteps);
  if (st != SWEPT_OK || nsteps == 0) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const Geom2& g = h->g;
  if (h->persistent) {
    if (nsteps / g.h + 1 > INT32_MAX) return fail(h, SWEPT_EINVAL, "nsteps too large for the persistent counters");
    if (!h->persist_blocks) {
      const int per_sm = h->value_bytes == 8 ? persist_blocks_per_sm_t<double>(h) : persist_blocks_per_sm_t<float>(h);
      if (per_sm < 1 || h->sm_count < 1) return fail(h, SWEPT_EINVAL, "persistent kernel does not fit on an SM");
      h->persist_blocks = per_sm * h->sm_count;
    }
    return run_graph(h, key_of("swept2d_persist", u_dev, nsteps), s, [&](cudaStream_t cs) {
      return h->value_bytes == 8 ? issue_persist_t<double>(h, (double*)u_dev, nsteps, cs)
                                 : issue_persist_t<float>(h, (float*)u_dev, nsteps, cs);
    });
  }
  const int64_t L = swept2d::launch_count2d(g, nsteps);
  const int64_t q = nsteps / g.h;
  const int64_t K = 256;  // half cycles per cached body graph (even: the body repeats with the tiling parity)
  const int64_t reps = q > 1 ? (q - 1) / K : 0;
  if (reps == 0)
    return run_graph(h, key_of("swept2d", u_dev, nsteps), s,
                     [&](cudaStream_t cs) { return issue_swept(h, u_dev, nsteps, 0, L, cs); });
  // head (the first pyramid), reps bodies of K half cycles (launches 1 .. 2K),
  // tail (the rest, including the last octahedron and the remainder)
  st = run_graph(h, key_of("swept2d_head", u_dev, 0), s,
                 [&](cudaStream_t cs) { return issue_swept(h, u_dev, nsteps, 0, 1, cs); });
  for (int64_t r = 0; r < reps && st == SWEPT_OK; ++r)
    st = run_graph(h, key_of("swept2d_body", nullptr, K), s,
                   [&](cudaStream_t cs) { return issue_swept(h, u_dev, nsteps, 1, 1 + 2 * K, cs); });
  if (st != SWEPT_OK) return st;
  const int64_t t0 = 1 + 2 * K * reps;
  return run_graph(h, key_of("swept2d_tail", u_dev, nsteps), s,
                   [&](cudaStream_t cs) { return issue_swept(h, u_dev, nsteps, t0, L, cs); });
}

swept_status classic2d_step_n(swept2d_handle* h, void* u_dev, int64_t nsteps, void* stream) {
  const swept_trace::Range trace_range("classic2d_step_n");
  swept_status st = check_ready(h, u_dev, nsteps);
  if (st != SWEPT_OK || nsteps == 0) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t kBody = 512;  // even, so a body starts and ends in u
  const int64_t reps = nsteps > 2 * kBody ? nsteps / kBody - 1 : 0;
  for (int64_t r = 0; r < reps && st == SWEPT_OK; ++r)
    st = run_graph(h, key_of("classic2d_body", u_dev, kBody), s,
                   [&](cudaStream_t cs) { return issue_classic(h, u_dev, 0, kBody, kBody, cs); });
  if (st != SWEPT_OK) return st;
  const int64_t rest = nsteps - reps * kBody;
  return run_graph(h, key_of("classic2d_tail", u_dev, rest), s,
                   [&](cudaStream_t cs) { return issue_classic(h, u_dev, 0, rest, rest, cs); });
}

swept_status swept2d_get_plan(const swept2d_handle* h, swept2d_plan_info* out) {
  if (!h || !out) return SWEPT_EINVAL;
  memset(out, 0, sizeof(*out));
  out->tile_w = h->g.W;
  out->threads = h->threads;
  out->half_cycle = h->g.h;
  out->persistent = h->persistent ? 1 : 0;
  out->tiles_x = h->g.ntx;
  out->tiles_y = h->g.nty;
  out->smem_bytes = (int64_t)h->smem;
  out->workspace_bytes = (int64_t)h->ws_bytes;
  return SWEPT_OK;
}

swept_status swept2d_check_schedule(swept2d_handle* h, int64_t nsteps, int64_t* computed) {
  if (!h || nsteps < 0) return SWEPT_EINVAL;
  std::string err;
  if ((double)(nsteps + 1) * (double)(h->g.nx * h->g.ny) > 2e8)
    return fail(h, SWEPT_EINVAL, "schedule check too large ((nsteps + 1) * nx * ny > 2e8)");
  if (h->persistent && swept2d::persist2d_items(h->g, nsteps) > 16384)
    return fail(h, SWEPT_EINVAL, "persistent schedule check too large (more than 16384 items)");
  if (!swept2d::check_schedule2d(h->g, nsteps, h->persistent, h->check_drop_wait, computed, &err))
    return fail(h, SWEPT_EDEVICE, err);
  return SWEPT_OK;
}

swept_status swept2d_set_option(swept2d_handle* h, int32_t option, int64_t value) {
  if (!h) return SWEPT_EINVAL;
  if (option == SWEPT_OPT_SPIN_LIMIT) {
    if (value < 1 || value > 0xffffffffLL) return fail(h, SWEPT_EINVAL, "spin limit outside [1, 2^32)");
    h->spin_limit = (uint32_t)value;
  } else if (option == SWEPT_OPT_START_ITEM) {
    if (value < 0) return fail(h, SWEPT_EINVAL, "start item < 0");
    h->start_item = value;
  } else if (option == SWEPT2D_OPT_CHECK_DROP_WAIT) {
    if (value < -1) return fail(h, SWEPT_EINVAL, "item < -1");
    h->check_drop_wait = value;
  } else {
    return fail(h, SWEPT_EINVAL, "unknown option");
  }
  drop_graphs(h);  // captured persistent launches carry the options
  return SWEPT_OK;
}

swept_status swept2d_sync_status(swept2d_handle* h, void* stream) {
  if (!h) return SWEPT_EINVAL;
  if (!h->ws) return fail(h, SWEPT_ENOWORKSPACE, "no workspace bound");
  const cudaStream_t s = (cudaStream_t)stream;
  int32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, h->ws + h->off_status, sizeof word, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->off_status, 0, sizeof word, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "swept2d_sync_status");
  if (word == 0) return SWEPT_OK;
  return fail(h, word == SWEPT_ETIMEOUT ? SWEPT_ETIMEOUT : SWEPT_EDEVICE, "device-side error word set");
}

swept_status swept2d_last_error(const swept2d_handle* h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return SWEPT_EINVAL;
  snprintf(buf, len, "%s", h->err.c_str());
  return SWEPT_OK;
}

void swept2d_free(swept2d_handle* h) {
  if (!h) return;
  drop_graphs(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

}  // extern "C"
