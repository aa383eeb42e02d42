// inst_fp16.cu -- kernels and launchers for storage type __half, arithmetic float.
#include "ops_impl.cuh"

namespace axl {
const Ops ops_fp16 = make_ops<__half, float>();
}  // namespace axl
