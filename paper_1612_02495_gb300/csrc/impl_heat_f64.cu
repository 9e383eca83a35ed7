// Heat (FTCS, Eq. HeatDisc): the kernels' FP64 instantiation (with its adjoint).
#include "impl_heat.cuh"

namespace swept {

const SchemeImpl* heat_impl_f64() {
  static const SchemeImpl k = make_heat_f64();
  return &k;
}

const SchemeImpl* heat_impl(int dtype) { return dtype == 0 ? heat_impl_f32() : heat_impl_f64(); }

}  // namespace swept
