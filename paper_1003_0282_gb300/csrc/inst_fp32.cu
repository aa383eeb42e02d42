// inst_fp32.cu -- kernels and launchers for storage type float, arithmetic float.
#include "ops_impl.cuh"

namespace axl {
const Ops ops_fp32 = make_ops<float, float>();
}  // namespace axl
