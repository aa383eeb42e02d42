// lattice.cuh -- velocity sets, weights and storage codecs of the GPU path.
//
// D2Q9 (Eq. 6) in (r, z) components: 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0),
// 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1); w = 4/9, 1/9, 1/36.
// D2Q4 (Eq. 53): 0 (1,0), 1 (0,1), 2 (-1,0), 3 (0,-1); weight 1/4.
// The numbering inside each group is not fixed by the paper; this one is
// the library's and is part of its ABI (include/axlbm.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace axl {

__host__ __device__ constexpr int cr9(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cz9(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
// index of the D2Q9 velocity with components (x, z)
__host__ __device__ constexpr int idx9(int x, int z) {
    return x == 0 ? (z == 0 ? 0 : (z > 0 ? 2 : 4))
                  : (x > 0 ? (z == 0 ? 1 : (z > 0 ? 5 : 8)) : (z == 0 ? 3 : (z > 0 ? 6 : 7)));
}
__host__ __device__ constexpr int opp9(int a) { return idx9(-cr9(a), -cz9(a)); }
__host__ __device__ constexpr double w9(int a) {
    return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

__host__ __device__ constexpr int cr4(int q) { return q == 0 ? 1 : (q == 2 ? -1 : 0); }
__host__ __device__ constexpr int cz4(int q) { return q == 1 ? 1 : (q == 3 ? -1 : 0); }
__host__ __device__ constexpr int opp4(int q) { return (q + 2) & 3; }
__host__ __device__ constexpr int idx4(int x, int z) {
    return x > 0 ? 0 : (x < 0 ? 2 : (z > 0 ? 1 : 3));
}

// Storage codecs: the stored value is a deviation from the rest state; the
// collision works in R (double or float).
template <class S>
struct Codec;
template <>
struct Codec<double> {
    __device__ static double load(const double* p) { return *p; }
    __device__ static void store(double* p, double v) { *p = v; }
};
template <>
struct Codec<float> {
    __device__ static float load(const float* p) { return *p; }
    __device__ static void store(float* p, float v) { *p = v; }
};
template <>
struct Codec<__half> {
    __device__ static float load(const __half* p) { return __half2float(*p); }
    __device__ static void store(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Codec<__nv_bfloat16> {
    __device__ static float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

}  // namespace axl
