// C-ABI runtime of a grid split over ranks (include/swept_slab.h): the plan,
// the rank's slab and workspace layout, and its launches.  The transfers
// between launches come from slab_plan.h and are carried out by the caller.
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "runtime.h"
#include "slab_plan.h"
#include "swept_slab.h"
#include "trace.h"

using swept::Geom;
using swept::Slab;

struct swept_slab {
  swept_config cfg;
  Geom g;
  Slab sl;
  const swept::SchemeImpl* impl = nullptr;
  unsigned char k[swept::KBYTES];
  int threads = 0;
  size_t smem = 0;
  int device = -1;
  int rank = 0, nranks = 1;
  size_t ebytes = 0;  // bytes of one edge buffer (aligned)
  char* ws = nullptr;
  size_t ws_bound = 0;
  bool prepared = false;
  std::string err;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

swept_status fail(swept_slab* h, swept_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

}  // namespace

namespace swept {

// The plan of swept_init for cfg, and the slab of `rank`: shared with the
// symbolic replay (check.cpp) so both see the same tiling.
swept_status slab_plan(const swept_config* cfg, int rank, int nranks, Geom* g, Slab* sl, swept_handle** plan_out) {
  if (!cfg || nranks < 1 || rank < 0 || rank >= nranks) return SWEPT_EINVAL;
  if (cfg->persistent != 0 || cfg->cluster != 0) return SWEPT_EUNSUPPORTED;
  swept_handle* h = nullptr;
  const swept_status st = swept_init(cfg, &h);
  if (st != SWEPT_OK) return st;
  if (!h->tiled) {
    swept_free(h);
    return SWEPT_EUNSUPPORTED;
  }
  if (nranks > h->g.nt) {
    swept_free(h);
    return SWEPT_EINVAL;
  }
  *g = h->g;
  *sl = make_slab(h->g, rank, nranks);
  if (plan_out)
    *plan_out = h;
  else
    swept_free(h);
  return SWEPT_OK;
}

}  // namespace swept

extern "C" {

swept_status swept_slab_init(const swept_config* cfg, int32_t rank, int32_t nranks, swept_slab** out) {
  if (!out) return SWEPT_EINVAL;
  *out = nullptr;
  Geom g;
  Slab sl;
  swept_handle* ph = nullptr;
  const swept_status st = swept::slab_plan(cfg, rank, nranks, &g, &sl, &ph);
  if (st != SWEPT_OK) return st;
  swept_slab* h = new (std::nothrow) swept_slab();
  if (!h) {
    swept_free(ph);
    return SWEPT_EINVAL;
  }
  h->cfg = *cfg;
  h->g = g;
  h->sl = sl;
  h->impl = ph->impl;
  memcpy(h->k, ph->k, sizeof(h->k));
  h->threads = ph->threads;
  h->smem = ph->smem;
  h->device = ph->device;
  h->rank = rank;
  h->nranks = nranks;
  h->ebytes = align_up((size_t)swept::slab_edge_values(g, sl) * h->impl->value_bytes);
  swept_free(ph);
  *out = h;
  return SWEPT_OK;
}

swept_status swept_slab_get_layout(const swept_slab* h, swept_slab_layout* out) {
  if (!h || !out) return SWEPT_EINVAL;
  const int64_t vb = h->impl->value_bytes;
  out->first_block = h->sl.b0;
  out->blocks = h->sl.nb;
  out->x0 = h->sl.x0;
  out->x1 = swept::slab_end(h->g, h->sl);
  out->state_len = h->sl.ul;
  out->edge_values = swept::slab_edge_values(h->g, h->sl);
  out->e0_offset = 0;
  out->e1_offset = (int64_t)h->ebytes / vb;
  out->workspace_bytes = (int64_t)(2 * h->ebytes);
  out->tile_w = h->g.W;
  out->threads = h->threads;
  out->half_cycle = h->g.h;
  out->value_bytes = (int32_t)vb;
  return SWEPT_OK;
}

swept_status swept_slab_bind_workspace(swept_slab* h, void* ws_dev, size_t bytes) {
  if (!h) return SWEPT_EINVAL;
  if (!ws_dev || ((uintptr_t)ws_dev % kAlign) != 0) return fail(h, SWEPT_EINVAL, "workspace NULL or not 256-byte aligned");
  if (bytes < 2 * h->ebytes) return fail(h, SWEPT_ENOMEM_WORKSPACE, "workspace smaller than the layout's workspace_bytes");
  h->ws = (char*)ws_dev;
  h->ws_bound = bytes;
  return SWEPT_OK;
}

swept_status swept_slab_launch_count(const swept_slab* h, int64_t nsteps, int64_t* count) {
  if (!h || !count || nsteps < 0) return SWEPT_EINVAL;
  *count = swept::launch_total(h->g, nsteps * h->g.S);
  return SWEPT_OK;
}

swept_status swept_slab_launch(swept_slab* h, void* u_dev, int64_t nsteps, int64_t i, void* stream) {
  const swept_trace::Range trace_range("swept_slab_launch");
  if (!h) return SWEPT_EINVAL;
  if (!u_dev || nsteps < 0) return fail(h, SWEPT_EINVAL, "u_dev is NULL or nsteps < 0");
  if (!h->ws) return fail(h, SWEPT_ENOWORKSPACE, "no workspace bound (swept_slab_bind_workspace)");
  const int64_t n_sub = nsteps * h->g.S;
  if (i < 0 || i >= swept::launch_total(h->g, n_sub)) return fail(h, SWEPT_EINVAL, "launch index out of range");
  if (h->device < 0) return fail(h, SWEPT_ECUDA, "no CUDA device was available when the handle was created");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(h, SWEPT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != h->device) return fail(h, SWEPT_EINVAL, "current device differs from the handle's device");
  if (!h->prepared) {
    if (h->smem > 48 * 1024) {
      e = h->impl->slab_prepare(h->smem);
      if (e != cudaSuccess)
        return fail(h, SWEPT_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
    h->prepared = true;
  }
  void* eb[2] = {h->ws, h->ws + h->ebytes};
  const swept::LaunchDesc d = swept::launch_at(h->g, n_sub, i);
  const cudaStream_t s = (cudaStream_t)stream;
  if (d.kind == 0)
    e = h->impl->slab_up(h->g, h->sl, h->k, u_dev, u_dev, eb[d.eout], d.hh, d.mode == swept::MODE_GAP ? 1 : 0,
                         h->threads, h->smem, s);
  else
    e = h->impl->slab_diamond(h->g, h->sl, h->k, u_dev, eb[d.ein], eb[d.eout], d.odd, d.mode, d.hh, h->threads,
                              h->smem, s);
  if (e != cudaSuccess) return fail(h, SWEPT_ECUDA, std::string("slab launch: ") + cudaGetErrorString(e));
  return SWEPT_OK;
}

swept_status swept_slab_xfers(const swept_slab* h, int64_t nsteps, int64_t i, swept_slab_xfer* out, int32_t cap,
                              int32_t* n) {
  if (!h || !n || nsteps < 0 || cap < 0 || (cap > 0 && !out)) return SWEPT_EINVAL;
  swept::Xfer x[swept::kMaxXfers];
  const int m = swept::slab_xfers(h->g, h->sl, nsteps * h->g.S, i, x);
  if (m > cap) return SWEPT_EINVAL;
  for (int j = 0; j < m; ++j) {
    out[j].peer = x[j].peer;
    out[j].recv = x[j].recv;
    out[j].region = x[j].region;
    out[j].reserved = 0;
    out[j].offset = x[j].offset;
    out[j].count = x[j].count;
  }
  *n = m;
  return SWEPT_OK;
}

swept_status swept_slab_last_error(const swept_slab* h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return SWEPT_EINVAL;
  snprintf(buf, len, "%s", h->err.c_str());
  return SWEPT_OK;
}

void swept_slab_free(swept_slab* h) { delete h; }

}  // extern "C"
