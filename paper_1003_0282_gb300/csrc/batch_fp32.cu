// batch_fp32.cu -- batch kernels and launchers for storage type float, arithmetic float.
#include "batch_ops.cuh"

namespace axl {
const BatchOps batch_ops_fp32 = make_batch_ops<float, float>();
}  // namespace axl
