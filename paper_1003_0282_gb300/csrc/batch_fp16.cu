// batch_fp16.cu -- batch kernels and launchers for storage type __half, arithmetic float.
#include "batch_ops.cuh"

namespace axl {
const BatchOps batch_ops_fp16 = make_batch_ops<__half, float>();
}  // namespace axl
