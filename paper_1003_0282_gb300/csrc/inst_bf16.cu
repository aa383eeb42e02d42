// inst_bf16.cu -- kernels and launchers for storage type __nv_bfloat16, arithmetic float.
#include "ops_impl.cuh"

namespace axl {
const Ops ops_bf16 = make_ops<__nv_bfloat16, float>();
}  // namespace axl
