// k_f64.cu -- kernel instantiations for populations stored as double.
#include "lbf_ops.cuh"

namespace lbf {
Ops *make_ops_f64(int dim) {
  if (dim == 2) return new OpsImpl<2, double>();
  return new OpsImpl<3, double>();
}
}  // namespace lbf
