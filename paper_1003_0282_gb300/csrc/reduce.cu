// reduce.cu -- final, fixed-order step of the check-step reductions.
//
// The step kernels leave one partial (max |d|u||, sum f, sum rho u_r / r,
// non-finite count) per thread block in the handle's scratch area; this one
// block folds them in a fixed order, so the FP64 sums are reproducible run to
// run for a given launch shape.
#include "internal.h"
#include "ops_impl.cuh"

namespace axl {

__global__ void __launch_bounds__(kThreads) k_finalize(const double* partials, int n, double* result) {
    Red v{0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        v.rmax = fmax(v.rmax, partials[4 * i + 0]);
        v.mass += partials[4 * i + 1];
        v.budget += partials[4 * i + 2];
        v.bad += partials[4 * i + 3];
    }
    block_reduce_store(v, result);
}

cudaError_t launch_finalize(const double* partials, int n, double* result, cudaStream_t stream) {
    k_finalize<<<1, kThreads, 0, stream>>>(partials, n, result);
    return cudaGetLastError();
}

}  // namespace axl
