// inst_w4.cu -- kernel instantiations for w = 4 components (real and complex).
#include "kernels.cuh"

namespace mpk {
const Ops* ops_w4(int cp) {
  static const Ops real_ops = Launch<4, 1>::table();
  static const Ops cplx_ops = Launch<4, 2>::table();
  return cp == 1 ? &real_ops : &cplx_ops;
}
}  // namespace mpk
