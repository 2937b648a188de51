// inst_w1.cu -- kernel instantiations for w = 1 components (real and complex).
#include "kernels.cuh"

namespace mpk {
const Ops* ops_w1(int cp) {
  static const Ops real_ops = Launch<1, 1>::table();
  static const Ops cplx_ops = Launch<1, 2>::table();
  return cp == 1 ? &real_ops : &cplx_ops;
}
}  // namespace mpk
