// inst_w3.cu -- kernel instantiations for w = 3 components (real and complex).
#include "kernels.cuh"

namespace mpk {
const Ops* ops_w3(int cp) {
  static const Ops real_ops = Launch<3, 1>::table();
  static const Ops cplx_ops = Launch<3, 2>::table();
  return cp == 1 ? &real_ops : &cplx_ops;
}
}  // namespace mpk
