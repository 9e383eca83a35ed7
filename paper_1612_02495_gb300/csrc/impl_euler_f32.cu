// 1D Euler (MUSCL-minmod + Rusanov + SSP-RK2): the kernels' FP32 instantiation.
#include "impl_euler.cuh"

namespace swept {

const SchemeImpl* euler_impl_f32() {
  static const SchemeImpl k = make_euler<float>();
  return &k;
}

}  // namespace swept
