// inst_w2.cu -- kernel instantiations for w = 2 components (real and complex).
#include "kernels.cuh"

namespace mpk {
const Ops* ops_w2(int cp) {
  static const Ops real_ops = Launch<2, 1>::table();
  static const Ops cplx_ops = Launch<2, 2>::table();
  return cp == 1 ? &real_ops : &cplx_ops;
}
}  // namespace mpk
