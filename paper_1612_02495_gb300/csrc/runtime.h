// Handle state shared by the runtime (api.cu) and the host schedule checker
// (check.cpp).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "swept.h"
#include "impl.h"

struct swept_handle {
  swept_config cfg;
  swept::Geom g;
  const swept::SchemeImpl* impl = nullptr;
  unsigned char k[swept::KBYTES];
  int threads = 0;
  size_t smem = 0;
  int device = 0;
  int sm_count = 0;
  // workspace (caller-owned device memory)
  char* ws = nullptr;
  size_t ws_bytes = 0;   // required
  size_t ws_bound = 0;   // bound size
  size_t off_e0 = 0, off_e1 = 0, off_tmp = 0, off_status = 0;
  size_t off_persist = 0;  // nt tile counters, then queue counter and error word
  bool tiled = true;  // false: the grid is too small for a swept tiling (classic only)
  bool persistent = false;
  bool cluster = false;
  int persist_blocks = 0;  // co-resident blocks of the persistent kernel (0 = not yet queried)
  uint32_t spin_limit = 1u << 24;  // polls a persistent block waits for an input tile (swept_set_option)
  int64_t start_item = 0;          // first queue item the persistent kernel claims (swept_set_option)
  // CUDA graphs cached by key; captured on a private stream
  cudaStream_t cap = nullptr;
  std::map<std::string, cudaGraphExec_t> graphs;
  std::string err;
  // last swept_forward_ckpt: its checkpoints (and the recorded tape of its last
  // segment) are what swept_adjoint(u0 = NULL) continues from
  const void* fwd_ckpt = nullptr;
  int64_t fwd_nsteps = -1;
  size_t fwd_bytes = 0;
  bool fwd_tape_valid = false;
};

namespace swept {
// symbolic replay of the swept launch sequence (check.cpp)
swept_status check_schedule(swept_handle* h, int64_t nsteps, int64_t* computed);
}  // namespace swept
