// Kuramoto-Sivashinsky (Eq. KSDisc + midpoint RK2):
// the scheme's constants and launch-table builders, shared by the FP32 and
// FP64 translation units (impl_ks_f32.cu, impl_ks_f64.cu), which compile in
// parallel.
#pragma once
#include "impl_common.cuh"

namespace swept {
namespace {

// c_a = 1/(4 dx), c_2 = 1/dx^2, c_4 = nu/dx^4, -dt/2, -dt: computed in double, rounded to T.
template <typename T>
void ks_consts(const double* param, double dx, double dt, void* kbuf) {
  typename KsOp<T>::K k;
  const double idx2 = 1.0 / (dx * dx);
  k.ca = (T)(1.0 / (4.0 * dx));
  k.c2 = (T)idx2;
  k.c4 = (T)(param[0] * (idx2 * idx2));
  k.mdth = (T)(-0.5 * dt);
  k.mdt = (T)(-dt);
  memcpy(kbuf, &k, sizeof(k));
}

// adjoint: 2 c_a, c_2, c_4, -dt, -dt/2, and -dt k4, -(dt/2) k4 with k4 = 1/dx^4 = dc_4/dnu
void ks_adj_consts(const double* param, double dx, double dt, void* kbuf) {
  KsAdjOp<double>::K k;
  const double idx2 = 1.0 / (dx * dx);
  const double k4 = idx2 * idx2;
  k.ca2 = 2.0 * (1.0 / (4.0 * dx));
  k.c2 = idx2;
  k.c4 = param[0] * k4;
  k.mdt = -dt;
  k.mdth = -0.5 * dt;
  k.mdtk4 = -dt * k4;
  k.mdthk4 = -0.5 * dt * k4;
  memcpy(kbuf, &k, sizeof(k));
}

template <typename T>
SchemeImpl make_ks() {
  using L = Launch<T, KsOp<T>>;
  SchemeImpl im{2, 2, 1, (int)sizeof(T), ks_consts<T>, L::smem_values, L::prepare, L::up, L::diamond,
                L::classic, L::copy, L::persist, L::persist_blocks_per_sm, L::cluster, L::up_tape, L::diamond_tape, nullptr,
                nullptr, nullptr, nullptr};
  im.slab_prepare = L::slab_prepare;
  im.slab_up = L::slab_up;
  im.slab_diamond = L::slab_diamond;
  return im;
}

SchemeImpl make_ks_f64() {
  using A = AdjLaunch<double, KsAdjOp<double>>;
  SchemeImpl im = make_ks<double>();
  im.make_adj_consts = ks_adj_consts;
  im.adj_prepare = A::prepare;
  im.adj_up = A::up;
  im.adj_diamond = A::diamond;
  return im;
}

}  // namespace
}  // namespace swept
