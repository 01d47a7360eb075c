// k_f32.cu -- kernel instantiations for populations stored as float.
#include "lbf_ops.cuh"

namespace lbf {
Ops *make_ops_f32(int dim) {
  if (dim == 2) return new OpsImpl<2, float>();
  return new OpsImpl<3, float>();
}
}  // namespace lbf
