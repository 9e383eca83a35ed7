// Kuramoto-Sivashinsky (Eq. KSDisc + midpoint RK2): the kernels' FP64 instantiation (with its adjoint).
#include "impl_ks.cuh"

namespace swept {

const SchemeImpl* ks_impl_f64() {
  static const SchemeImpl k = make_ks_f64();
  return &k;
}

const SchemeImpl* ks_impl(int dtype) { return dtype == 0 ? ks_impl_f32() : ks_impl_f64(); }

}  // namespace swept
