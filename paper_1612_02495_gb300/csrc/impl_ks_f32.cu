// Kuramoto-Sivashinsky (Eq. KSDisc + midpoint RK2): the kernels' FP32 instantiation.
#include "impl_ks.cuh"

namespace swept {

const SchemeImpl* ks_impl_f32() {
  static const SchemeImpl k = make_ks<float>();
  return &k;
}

}  // namespace swept
