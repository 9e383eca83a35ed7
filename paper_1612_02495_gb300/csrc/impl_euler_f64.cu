// 1D Euler (MUSCL-minmod + Rusanov + SSP-RK2): the kernels' FP64 instantiation.
#include "impl_euler.cuh"

namespace swept {

const SchemeImpl* euler_impl_f64() {
  static const SchemeImpl k = make_euler<double>();
  return &k;
}

const SchemeImpl* euler_impl(int dtype) { return dtype == 0 ? euler_impl_f32() : euler_impl_f64(); }

}  // namespace swept
