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

// Fixed-order fold of every domain's tile partials (and ring values after an
// odd step) into result[d][4] = {max |d|u||, mass, budget, non-finite count}.
__global__ void __launch_bounds__(kThreads)
k_domain_fold(const int* tile_start, const int* tile_index, const double* tile_part, const int* ring_start,
              const double* ring_part, int with_ring, double* result) {
    const int d = blockIdx.x;
    Red v{0.0, 0.0, 0.0, 0.0};
    for (int i = tile_start[d] + threadIdx.x; i < tile_start[d + 1]; i += blockDim.x) {
        const double* p = tile_part + 4ll * tile_index[i];
        v.rmax = fmax(v.rmax, p[0]);
        v.mass += p[1];
        v.budget += p[2];
        v.bad += p[3];
    }
    if (with_ring) {
        for (int i = ring_start[d] + threadIdx.x; i < ring_start[d + 1]; i += blockDim.x) {
            const double* p = ring_part + 4ll * i;
            v.rmax = fmax(v.rmax, p[0]);
            v.mass += p[1];
            v.budget += p[2];
            v.bad += p[3];
        }
    }
    block_reduce_store(v, result + 4ll * d);
}

cudaError_t launch_domain_fold(int ndom, const int* tile_start, const int* tile_index, const double* tile_part,
                               const int* ring_start, const double* ring_part, int with_ring, double* result,
                               cudaStream_t stream) {
    k_domain_fold<<<ndom, kThreads, 0, stream>>>(tile_start, tile_index, tile_part, ring_start, ring_part, with_ring,
                                                 result);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int n, double* result, cudaStream_t stream) {
    k_finalize<<<1, kThreads, 0, stream>>>(partials, n, result);
    return cudaGetLastError();
}

}  // namespace axl
