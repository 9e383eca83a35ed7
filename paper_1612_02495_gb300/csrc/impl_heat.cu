// Heat (FTCS, Eq. HeatDisc) instantiation of the swept and classic kernels.
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

template <typename T>
SchemeImpl make_heat() {
  using L = Launch<T, HeatOp<T>>;
  return SchemeImpl{1, 1, 1, (int)sizeof(T), heat_consts<T>, L::smem_values, L::prepare, L::up, L::diamond,
                    L::classic, L::copy};
}

const SchemeImpl kHeatF32 = make_heat<float>();
const SchemeImpl kHeatF64 = make_heat<double>();

}  // namespace

const SchemeImpl* heat_impl(int dtype) { return dtype == 0 ? &kHeatF32 : &kHeatF64; }

}  // namespace swept
