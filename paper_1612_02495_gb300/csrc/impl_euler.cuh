// 1D Euler (MUSCL-minmod + Rusanov + SSP-RK2):
// the scheme's constants and launch-table builders, shared by the FP32 and
// FP64 translation units (impl_euler_f32.cu, impl_euler_f64.cu), which compile in
// parallel.
#pragma once
#include "impl_common.cuh"

namespace swept {
namespace {

// gamma, gamma - 1, 1/(gamma - 1), -dt/dx: computed in double, rounded to T.
template <typename T>
void euler_consts(const double* param, double dx, double dt, void* kbuf) {
  typename EulerOp<T>::K k;
  k.gamma = (T)param[0];
  k.gm1 = (T)(param[0] - 1.0);
  k.igm1 = (T)(1.0 / (param[0] - 1.0));
  k.mdtdx = (T)(-(dt / dx));
  memcpy(kbuf, &k, sizeof(k));
}

template <typename T>
cudaError_t euler_classic(const Geom& g, const void* kb, int stage, const void* in, void* out, cudaStream_t s) {
  const int B = 256;
  const unsigned grid = (unsigned)((g.N + B - 1) / B);
  const size_t smem = sizeof(T) * (3 * (B + 4) + 3 * (B + 1));
  const auto k = Launch<T, EulerOp<T>>::kc(kb);
  // B cells per block and one more warp, so that each of the B + 1 faces
  // has its own thread
  if (stage == 0)
    k_classic_euler<T, 0><<<grid, B + 32, smem, s>>>(g.N, g.bc, k, (const T*)in, (T*)out, B);
  else
    k_classic_euler<T, 1><<<grid, B + 32, smem, s>>>(g.N, g.bc, k, (const T*)in, (T*)out, B);
  return cudaGetLastError();
}

template <typename T>
SchemeImpl make_euler() {
  using L = Launch<T, EulerOp<T>>;
  SchemeImpl im{2, 2, 3, (int)sizeof(T), euler_consts<T>, L::smem_values, L::prepare, L::up, L::diamond,
                euler_classic<T>, L::copy, L::persist, L::persist_blocks_per_sm, L::cluster, L::up_tape, L::diamond_tape, nullptr,
                nullptr, nullptr, nullptr};
  im.slab_prepare = L::slab_prepare;
  im.slab_up = L::slab_up;
  im.slab_diamond = L::slab_diamond;
  return im;
}

}  // namespace
}  // namespace swept
