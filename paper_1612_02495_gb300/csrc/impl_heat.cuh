// Heat (FTCS, Eq. HeatDisc):
// the scheme's constants and launch-table builders, shared by the FP32 and
// FP64 translation units (impl_heat_f32.cu, impl_heat_f64.cu), which compile in
// parallel.
#pragma once
#include "impl_common.cuh"

namespace swept {
namespace {

// Fo = alpha dt / dx^2 and 1 - 2 Fo, computed in double, then rounded to T.
template <typename T>
void heat_consts(const double* param, double dx, double dt, void* kbuf) {
  typename HeatOp<T>::K k;
  const double fo = (param[0] * dt) / (dx * dx);
  k.fo = (T)fo;
  k.c1 = (T)(1.0 - 2.0 * fo);
  memcpy(kbuf, &k, sizeof(k));
}

// adjoint: Fo, 1 - 2 Fo and dt / dx^2 (the derivative of Fo with respect to alpha)
void heat_adj_consts(const double* param, double dx, double dt, void* kbuf) {
  HeatAdjOp<double>::K k;
  const double fo = (param[0] * dt) / (dx * dx);
  k.fo = fo;
  k.c1 = 1.0 - 2.0 * fo;
  k.kk = dt / (dx * dx);
  memcpy(kbuf, &k, sizeof(k));
}

template <typename T>
SchemeImpl make_heat() {
  using L = Launch<T, HeatOp<T>>;
  SchemeImpl im{1, 1, 1, (int)sizeof(T), heat_consts<T>, L::smem_values, L::prepare, L::up, L::diamond,
                L::classic, L::copy, L::persist, L::persist_blocks_per_sm, L::cluster, L::up_tape, L::diamond_tape, nullptr,
                nullptr, nullptr, nullptr};
  im.slab_prepare = L::slab_prepare;
  im.slab_up = L::slab_up;
  im.slab_diamond = L::slab_diamond;
  return im;
}

SchemeImpl make_heat_f64() {
  using A = AdjLaunch<double, HeatAdjOp<double>>;
  SchemeImpl im = make_heat<double>();
  im.make_adj_consts = heat_adj_consts;
  im.adj_prepare = A::prepare;
  im.adj_up = A::up;
  im.adj_diamond = A::diamond;
  return im;
}

}  // namespace
}  // namespace swept
