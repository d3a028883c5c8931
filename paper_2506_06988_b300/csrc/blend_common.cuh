// blend_common.cuh -- the per-(pixel, Gaussian) evaluation shared by the
// forward and backward blending kernels.  Every operation uses an explicit
// rounding intrinsic, so the compiler cannot contract them differently in
// the two kernels: the backward pass replays exactly the decisions (3-sigma
// cut, alpha >= 1/255) the forward pass took.
#pragma once

#include "hm_internal.cuh"

namespace hm {

constexpr float kNegHalfLog2e = kConicScale;             // -log2(e)/2
constexpr float kQ3 = 9.0f * kNegHalfLog2e;                // q at d^2 = 9
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// q = K d^2 at pixel centre (fpx, fpy)
__device__ __forceinline__ float eval_q(const float4 &A, const float4 &B, float fpx, float fpy,
                                        float &dx, float &dy) {
    dx = __fsub_rn(fpx, A.x);
    dy = __fsub_rn(fpy, A.y);
    return __fmaf_rn(dx, __fmaf_rn(A.z, dx, __fmul_rn(A.w, dy)), __fmul_rn(__fmul_rn(B.x, dy), dy));
}

// The two pixels thread t owns: each warp covers a compact 8x8 block of the
// tile (lane l at column l % 8, rows l / 8 and l / 8 + 4), so a small
// Gaussian activates few warps.  Requires TW % 8 == 0 and TH % 8 == 0.
template <int TW>
__device__ __forceinline__ void pixel_pair(int t, int x0, int y0, int &px, int &pya, int &pyb) {
    constexpr int WX = TW / 8;                  // warps across the tile
    const int w = t >> 5, l = t & 31;
    px = x0 + (w % WX) * 8 + (l & 7);
    pya = y0 + (w / WX) * 8 + (l >> 3);
    pyb = pya + 4;
}

// q = K d^2 at two pixel centres of one column, (fpx, fpy.x) and (fpx, fpy.y),
// in packed FP32x2: dx is shared, K a dx^2 and 2K b dx once per Gaussian
// (eval_qcol), then q = K a dx^2 + dy (2K b dx + K c dy) for both pixels
// (eval_qrows; a thread with several pixel pairs of one column evaluates the
// column part once).
struct QCol {
    float dx, adx, bdx;
};
__device__ __forceinline__ QCol eval_qcol(const float4 &A, float fpx) {
    QCol c;
    c.dx = __fsub_rn(fpx, A.x);
    c.adx = __fmul_rn(__fmul_rn(A.z, c.dx), c.dx);
    c.bdx = __fmul_rn(A.w, c.dx);
    return c;
}
__device__ __forceinline__ float2 eval_qrows(const float4 &A, const float4 &B, const QCol &c, float2 fpy,
                                             float2 &dy) {
    dy = __fadd2_rn(fpy, make_float2(-A.y, -A.y));
    const float2 t = __ffma2_rn(make_float2(B.x, B.x), dy, make_float2(c.bdx, c.bdx));
    return __ffma2_rn(dy, t, make_float2(c.adx, c.adx));
}
__device__ __forceinline__ float2 eval_q2(const float4 &A, const float4 &B, float fpx, float2 fpy,
                                          float &dx, float2 &dy) {
    const QCol c = eval_qcol(A, fpx);
    dx = c.dx;
    return eval_qrows(A, B, c, fpy, dy);
}

// alpha = min(0.99, o 2^q) for both pixels; G = 2^q, araw = o G
__device__ __forceinline__ float2 eval_alpha2(float o, float2 q, float2 &G, float2 &araw) {
    G = make_float2(ex2_approx(q.x), ex2_approx(q.y));
    araw = __fmul2_rn(make_float2(o, o), G);
    return make_float2(fminf(kAlphaMax, araw.x), fminf(kAlphaMax, araw.y));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace hm
