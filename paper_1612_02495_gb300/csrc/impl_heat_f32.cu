// Heat (FTCS, Eq. HeatDisc): the kernels' FP32 instantiation.
#include "impl_heat.cuh"

namespace swept {

const SchemeImpl* heat_impl_f32() {
  static const SchemeImpl k = make_heat<float>();
  return &k;
}

}  // namespace swept
