// f32x2.cuh — two FP32 lanes per register pair: Blackwell's packed FP32
// instructions (add/mul/fma .rn.f32x2) through the CUDA builtins, so that the
// compiler allocates the register pairs itself.  The radiation kernels give
// each thread two adjacent directions and work on both at once.
#pragma once
#include <cuda_runtime.h>

struct F2 { float x, y; };
__device__ __forceinline__ F2 f2(float a) { return F2{a, a}; }
__device__ __forceinline__ float2 v2(F2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ F2 u2(float2 a) { return F2{a.x, a.y}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return u2(__fadd2_rn(v2(a), v2(b))); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return u2(__fadd2_rn(v2(a), make_float2(-b.x, -b.y))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return u2(__fmul2_rn(v2(a), v2(b))); }
// a * b + c
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return u2(__ffma2_rn(v2(a), v2(b), v2(c))); }

// min(|a|, |b|) carrying the sign sign(a) XOR sign(b): negative exactly when a
// and b have opposite signs (PTX min.xorsign.abs)
__device__ __forceinline__ float min_xorsign_abs(float a, float b) {
    float r;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Half of the monotonised central slope, sign(dl) min(|dl|, |dr|, |dl + dr|/4)
// where dl and dr have the same sign, 0 otherwise, from h = (dl + dr)/4:
// m = max(min_xorsign_abs(dl, dr), 0) is min(|dl|, |dr|) for equal signs and 0
// otherwise; min_xorsign_abs(h, m) then has magnitude min(|h|, m) and the sign
// of h (m >= 0), which is the sign of dl and dr when they agree.  Three
// min/max instructions per lane instead of the compare-and-select form.
__device__ __forceinline__ float mc_half_xs(float dl, float dr, float h) {
    const float m = fmaxf(min_xorsign_abs(dl, dr), 0.0f);
    return min_xorsign_abs(h, m);
}
__device__ __forceinline__ F2 mc_half2(F2 dl, F2 dr) {
    const F2 h = f2(0.25f) * (dl + dr);
    return F2{mc_half_xs(dl.x, dr.x, h.x), mc_half_xs(dl.y, dr.y, h.y)};
}
