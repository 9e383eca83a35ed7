// swept_step_n_static: the swept solve with its edge buffers in a fixed,
// file-scope device array instead of caller-bound workspace.
//
// For callers that cannot call cudaMalloc: code whose device memory is owned
// by an outside memory manager (an embedding application or framework that
// hands out every byte itself and forbids raw allocation), and hot loops that
// cannot afford the device-wide synchronisation cudaMalloc/cudaFree imply.
// This entry point allocates nothing, host or device: no handle, no CUDA
// graph, no stream, no cudaMalloc/cudaFree, no allocating library call.  The
// caller passes the state u_dev (input and output, updated in place).
//
// The scratch is one array of kStaticScratchBytes that every GPU loading this
// library keeps until the process exits.  All calls share it and it keeps the
// last call's contents; the swept passes write every edge value before reading
// it, so nothing has to start at zero.  Calls that overlap on the GPU (two
// streams, or two host threads) race on the array.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "impl.h"
#include "swept.h"
#include "swept_phases.cuh"

namespace {

constexpr size_t kStaticScratchBytes = SWEPT_STATIC_SCRATCH_BYTES;  // 8 MiB (include/swept.h)
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on each device.  In host code the name
// g_static_scratch is only a host-side stand-in, never a device address.
void* g_scratch_addr[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: look up the array's address.
cudaError_t scratch_on(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

const swept::SchemeImpl* pick(int scheme, int dtype) {
  if (dtype != SWEPT_F32 && dtype != SWEPT_F64) return nullptr;
  if (scheme == SWEPT_HEAT) return swept::heat_impl(dtype);
  if (scheme == SWEPT_KS) return swept::ks_impl(dtype);
  if (scheme == SWEPT_EULER) return swept::euler_impl(dtype);
  return nullptr;
}

}  // namespace

extern "C" swept_status swept_step_n_static(const swept_config* cfg, void* u_dev, int64_t nsteps, void* stream) {
  if (!cfg || !u_dev || nsteps < 0) return SWEPT_EINVAL;
  const swept::SchemeImpl* im = pick(cfg->scheme, cfg->dtype);
  if (!im) return SWEPT_EINVAL;
  if (cfg->bc != SWEPT_BC_PERIODIC && cfg->bc != SWEPT_BC_REFLECTIVE) return SWEPT_EINVAL;
  if (cfg->scheme == SWEPT_KS && cfg->bc != SWEPT_BC_PERIODIC) return SWEPT_EINVAL;
  if (!(cfg->dx > 0) || !(cfg->dt > 0) || cfg->n < 8) return SWEPT_EINVAL;
  if (cfg->scheme == SWEPT_EULER && !(cfg->param[0] > 1.0)) return SWEPT_EINVAL;
  const int R = im->R;
  const int W = cfg->tile_w;  // required here: no planning state is kept
  if (W < 4 * R || W % (4 * R) != 0 || cfg->n % W != 0 || cfg->n / W < 2) return SWEPT_EINVAL;
  const int threads = cfg->threads > 0 ? cfg->threads : (W >= 256 ? 256 : ((W + 31) / 32) * 32);
  if (threads < 32 || threads > 1024 || threads % 32 != 0) return SWEPT_EINVAL;

  swept::Geom g;
  g.N = cfg->n;
  g.W = W;
  g.R = R;
  g.S = im->S;
  g.C = im->C;
  g.h = W / (2 * R);
  g.M = W + 2 * R;
  g.nt = cfg->n / W;
  g.E = 2 * g.h * g.C * 2 * R;
  g.bc = cfg->bc;
  g.chunk = 1;
  const size_t ebytes = align_up((size_t)g.nt * g.E * im->value_bytes);
  if (2 * ebytes > kStaticScratchBytes) return SWEPT_ENOMEM_WORKSPACE;  // grid too large for the 8 MiB array
  if (nsteps == 0) return SWEPT_OK;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SWEPT_ECUDA;
  int max_smem = 0;
  if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return SWEPT_ECUDA;
  const size_t smem = (size_t)im->smem_values(g.M) * im->value_bytes;
  if (smem > (size_t)max_smem) return SWEPT_EINVAL;
  if (smem > 48 * 1024 && im->prepare(smem) != cudaSuccess) return SWEPT_ECUDA;  // raises only
  void* scratch = nullptr;
  if (scratch_on(dev, &scratch) != cudaSuccess) return SWEPT_ECUDA;
  void* eb[2] = {scratch, (char*)scratch + ebytes};

  unsigned char k[swept::KBYTES];
  im->make_consts(cfg->param, cfg->dx, cfg->dt, k);
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t err = cudaSuccess;
  swept::for_each_launch(g, nsteps * g.S, [&](int kind, int odd, int mode, int hh, int64_t pass) {
    if (err != cudaSuccess) return;
    if (kind == 0) {
      const int out = pass >= 0 ? (int)(pass & 1) : 0;
      err = im->up(g, k, u_dev, u_dev, eb[out], hh, mode == swept::MODE_GAP, threads, smem, s);
    } else {
      const int in = pass >= 1 ? (int)((pass - 1) & 1) : 0;
      const int out = pass >= 1 ? (int)(pass & 1) : 1;
      err = im->diamond(g, k, u_dev, eb[in], eb[out], odd, mode, hh, threads, smem, s);
    }
  });
  return err == cudaSuccess ? SWEPT_OK : SWEPT_ECUDA;
}
