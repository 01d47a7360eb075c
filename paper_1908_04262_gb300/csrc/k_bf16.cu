// k_bf16.cu -- kernel instantiations for populations stored as __nv_bfloat16.
#include "lbf_ops.cuh"

namespace lbf {
Ops *make_ops_bf16(int dim) {
  if (dim == 2) return new OpsImpl<2, __nv_bfloat16>();
  return new OpsImpl<3, __nv_bfloat16>();
}
}  // namespace lbf
