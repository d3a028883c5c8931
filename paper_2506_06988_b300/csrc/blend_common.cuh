// blend_common.cuh -- the per-(pixel, Gaussian) evaluation shared by the
// forward and backward blending kernels.  Every operation uses an explicit
// rounding intrinsic, so the compiler cannot contract them differently in
// the two kernels: the backward pass replays exactly the decisions (3-sigma
// cut, alpha >= 1/255) the forward pass took.
#pragma once

#include "hm_internal.cuh"

namespace hm {

constexpr float kNegHalfLog2e = -0.72134752044448170f;   // -log2(e)/2
constexpr float kQ3 = 9.0f * kNegHalfLog2e;                // q at d^2 = 9
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// staged record: conic pre-scaled by K = -log2(e)/2 so that
// q = K d^2 and G = exp(-d^2/2) = 2^q
struct Staged {
    float4 a;   // mean x, mean y, K*conic_xx, 2K*conic_xy
    float4 b;   // K*conic_yy, opacity, depth, -
    float4 c;   // r, g, b, -
};

__device__ __forceinline__ void stage_record(const Record &r, float4 &a, float4 &b, float4 &c) {
    a = make_float4(r.a.x, r.a.y, __fmul_rn(kNegHalfLog2e, r.a.z), __fmul_rn(2.f * kNegHalfLog2e, r.a.w));
    b = make_float4(__fmul_rn(kNegHalfLog2e, r.b.x), r.b.y, r.b.z, 0.f);
    c = r.c;
}

// q = K d^2 at pixel centre (fpx, fpy)
__device__ __forceinline__ float eval_q(const float4 &A, const float4 &B, float fpx, float fpy,
                                        float &dx, float &dy) {
    dx = __fsub_rn(fpx, A.x);
    dy = __fsub_rn(fpy, A.y);
    return __fmaf_rn(dx, __fmaf_rn(A.z, dx, __fmul_rn(A.w, dy)), __fmul_rn(__fmul_rn(B.x, dy), dy));
}

}  // namespace hm
