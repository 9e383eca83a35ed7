// Kuramoto-Sivashinsky (Eq. KSDisc + midpoint RK2) instantiation of the kernels.
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

template <typename T>
SchemeImpl make_ks() {
  using L = Launch<T, KsOp<T>>;
  return SchemeImpl{2, 2, 1, (int)sizeof(T), ks_consts<T>, L::smem_values, L::prepare, L::up, L::diamond,
                    L::classic, L::copy};
}

const SchemeImpl kKsF32 = make_ks<float>();
const SchemeImpl kKsF64 = make_ks<double>();

}  // namespace

const SchemeImpl* ks_impl(int dtype) { return dtype == 0 ? &kKsF32 : &kKsF64; }

}  // namespace swept
