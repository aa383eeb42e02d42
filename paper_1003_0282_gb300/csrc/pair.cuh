// pair.cuh -- arithmetic on a pair of FP32 values with Blackwell's paired
// FP32 instructions (add/mul/fma on f32x2), and the scalar overloads the
// collision code shares with it.
//
// The bulk kernel updates two nodes of the same radius (two rows of a tile)
// per thread; holding both in one F2 halves the arithmetic instructions.
#pragma once

#include <cuda_runtime.h>

namespace axl {

struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    F2 r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 r;
    r.v = __ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v);
    return r;
}
__device__ __forceinline__ F2 fmaR(F2 a, F2 b, F2 c) {
    F2 r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}
__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }

// Reciprocal: correctly rounded in FP32 (cheaper than a divide; products
// differ from true quotients by at most an ulp), a plain divide in FP64.
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ F2 rcp(F2 x) { return F2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }

template <class R>
struct ScalarOf {
    using type = R;
};
template <>
struct ScalarOf<F2> {
    using type = float;
};

}  // namespace axl
