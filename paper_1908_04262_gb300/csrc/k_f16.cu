// k_f16.cu -- kernel instantiations for populations stored as __half.
#include "lbf_ops.cuh"

namespace lbf {
Ops *make_ops_f16(int dim) {
  if (dim == 2) return new OpsImpl<2, __half>();
  return new OpsImpl<3, __half>();
}
}  // namespace lbf
