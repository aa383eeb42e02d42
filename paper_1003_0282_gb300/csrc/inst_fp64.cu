// inst_fp64.cu -- kernels and launchers for storage type double, arithmetic double.
#include "ops_impl.cuh"

namespace axl {
const Ops ops_fp64 = make_ops<double, double>();
}  // namespace axl
