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

// Reciprocal in FP32: the hardware estimate (PTX rcp.approx.ftz.f32, within
// about an ulp) refined by one Newton-Raphson step for 1/x, r' = r + r (1 -
// x r), which squares the estimate's relative error; the two fused
// multiply-adds leave the result within one ulp of 1/x (faithful rounding)
// for the normal arguments the collision takes (densities near rho0, radii
// of at least 1/2), without the branches of the correctly rounded call.  The
// scalar and the paired forms round alike, lane by lane.  FP64: a divide.
__device__ __forceinline__ float rcp_estimate(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp(float x) {
    const float r = rcp_estimate(x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ F2 rcp(F2 x) {
    const float2 r = make_float2(rcp_estimate(x.v.x), rcp_estimate(x.v.y));
    const float2 e = __ffma2_rn(make_float2(-x.v.x, -x.v.y), r, make_float2(1.0f, 1.0f));
    F2 out;
    out.v = __ffma2_rn(r, e, r);
    return out;
}

template <class R>
struct ScalarOf {
    using type = R;
};
template <>
struct ScalarOf<F2> {
    using type = float;
};

}  // namespace axl
