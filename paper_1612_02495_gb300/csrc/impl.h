// Per-(scheme, dtype) launch table, filled by one translation unit per scheme
// (impl_<scheme>_f32.cu / impl_<scheme>_f64.cu) and used by the runtime (api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "swept_geom.cuh"


namespace swept {

constexpr int KBYTES = 64;  // room for any scheme's constant struct

struct SchemeImpl {
  int R, S, C;
  int value_bytes;
  // constants of the scheme for this config, written into kbuf (<= KBYTES)
  void (*make_consts)(const double* param, double dx, double dt, void* kbuf);
  int64_t (*smem_values)(int M);
  // raise the dynamic shared-memory limit of the swept kernels to `bytes`
  cudaError_t (*prepare)(size_t bytes);
  cudaError_t (*up)(const Geom& g, const void* k, const void* u_in, void* u_out, void* e_out, int hh, int write_top,
                    int threads, size_t smem, cudaStream_t s);
  cudaError_t (*diamond)(const Geom& g, const void* k, void* u_out, const void* e_in, void* e_out, int odd, int mode,
                         int hh, int threads, size_t smem, cudaStream_t s);
  // one classic sub-timestep (stage 0 or 1) from `in` into `out`
  cudaError_t (*classic)(const Geom& g, const void* k, int stage, const void* in, void* out, cudaStream_t s);
  cudaError_t (*copy)(int64_t n, const void* src, void* dst, cudaStream_t s);
  // persistent single-problem kernel over n_sub sub-timesteps (grid = blocks)
  cudaError_t (*persist)(const Geom& g, const void* k, void* u, void* e0, void* e1, int64_t n_sub, int* done,
                         unsigned long long* queue, int* error, uint32_t spin_limit, int64_t start_item, int blocks,
                         int threads, size_t smem, cudaStream_t s);
  // co-resident blocks per SM of the persistent kernel (variant P = Geom::P)
  int (*persist_blocks_per_sm)(int P, int threads, size_t smem);
  // whole solve in one cluster of g.nt (<= 16) blocks, edges through DSMEM
  cudaError_t (*cluster)(const Geom& g, const void* k, void* u, int64_t n_sub, int threads, size_t smem,
                         cudaStream_t s);
  // forward passes that also record every tier into a tape (adjoint support;
  // nullptr for schemes without an adjoint)
  cudaError_t (*up_tape)(const Geom& g, const void* k, const void* u_in, void* u_out, void* e_out, int hh,
                         int write_top, int threads, size_t smem, void* tape, int64_t tier0, int64_t ntiers,
                         int64_t base, cudaStream_t s);
  cudaError_t (*diamond_tape)(const Geom& g, const void* k, void* u_out, const void* e_in, void* e_out, int odd,
                              int mode, int hh, int threads, size_t smem, void* tape, int64_t tier0, int64_t ntiers,
                              int64_t base, cudaStream_t s);
  // adjoint constants and passes (FP64 only; nullptr where there is no adjoint)
  void (*make_adj_consts)(const double* param, double dx, double dt, void* kbuf);
  cudaError_t (*adj_prepare)(size_t bytes);
  cudaError_t (*adj_up)(const Geom& g, const void* ka, const void* lam_in, void* lam_out, void* e_out, int hh,
                        int write_top, int threads, size_t smem, const void* tape, int64_t top, int64_t base,
                        double* slots, cudaStream_t s);
  cudaError_t (*adj_diamond)(const Geom& g, const void* ka, void* lam_out, const void* e_in, void* e_out, int odd,
                             int mode, int hh, int threads, size_t smem, const void* tape, int64_t top, int64_t base,
                             double* slots, cudaStream_t s);
  // one pass of a slab of a grid split over ranks (blocks [sl.b0, sl.b0 + sl.nb));
  // slab_prepare raises the slab kernels' shared-memory limit
  cudaError_t (*slab_prepare)(size_t bytes);
  cudaError_t (*slab_up)(const Geom& g, const Slab& sl, const void* k, const void* u_in, void* u_out, void* e_out,
                         int hh, int write_top, int threads, size_t smem, cudaStream_t s);
  cudaError_t (*slab_diamond)(const Geom& g, const Slab& sl, const void* k, void* u_out, const void* e_in,
                              void* e_out, int odd, int mode, int hh, int threads, size_t smem, cudaStream_t s);
};

// Raise kernel `fn`'s dynamic shared-memory limit on the current device to at
// least `bytes` (when bytes > 48 KB).  It never lowers the limit: every handle
// and every static call shares the kernel instantiations, so a smaller tile
// must not take away the opt-in a larger tile's handle set up earlier.  The
// read-check-set runs under one process-wide lock.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);

const SchemeImpl* heat_impl(int dtype);
const SchemeImpl* ks_impl(int dtype);
const SchemeImpl* euler_impl(int dtype);
const SchemeImpl* heat_impl_f32();
const SchemeImpl* heat_impl_f64();
const SchemeImpl* ks_impl_f32();
const SchemeImpl* ks_impl_f64();
const SchemeImpl* euler_impl_f32();
const SchemeImpl* euler_impl_f64();

}  // namespace swept
