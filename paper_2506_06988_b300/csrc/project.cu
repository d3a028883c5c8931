// project.cu -- Gaussian projection (Eq. 1; Sec. 3.1: Sigma = R S S^T R^T,
// Sigma' = J W Sigma W^T J^T) and view-dependent SH colour, per
// (camera, Gaussian), into 48-byte records.
//
// One thread per Gaussian loops over the cameras, so the parameters (236 B
// per Gaussian at SH degree 3) are read from HBM once per call whatever the
// number of views; the view-independent factor M = R(q) S is formed once.
//
// Numerics.
//  * The depth key is fp32(fma(R20, x, fma(R21, y, fma(R22, z, t2)))) in
//    FP64, bit-identical to the definition the sort and the mesh cut-off
//    rely on (4 FP64 operations per camera and Gaussian -- the FP64 pipe is
//    1/64 of the FP32 rate on B300).
//  * The view-space point used for the projection is a float-float
//    (TwoProduct/TwoSum) evaluation in FP32, and x/z, y/z take one residual
//    correction, so the projected mean carries close to FP32 rounding only.
//  * Sigma' is formed as V V^T with V = (J W)(R S) (2x3).  det(Sigma' + 0.3 I)
//    = |V0 x V1|^2 + 0.3 (|V0|^2 + |V1|^2) + 0.09 (Lagrange's identity) is a
//    sum of non-negative terms, with the cross product from FMA-based
//    differences of products and V0.V1 from a compensated dot product, so
//    the conic of a thin ellipse does not suffer the cancellation of
//    a c - b^2.
#include "hm_internal.cuh"
#include "hm_host.h"
#include "sh.cuh"

namespace hm {

namespace {

// a*b - c*d with one FMA-corrected rounding (Kahan)
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
    float cd = c * d;
    float err = fmaf(-c, d, cd);
    float dop = fmaf(a, b, -cd);
    return dop + err;
}

// compensated dot product of 3-vectors (TwoProduct + TwoSum)
__device__ __forceinline__ float dot3_c(const float *u, const float *v) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float p = u[k] * v[k];
        float pe = fmaf(u[k], v[k], -p);
        float t = s + p;
        float z = t - s;
        float se = (s - (t - z)) + (p - z);
        s = t;
        c += pe + se;
    }
    return s + c;
}

// r0 x + r1 y + r2 z + t as an unevaluated float-float sum (hi, lo):
// TwoProduct (FMA) for each product and TwoSum for each addition, so the
// pair carries the value to ~2^-46 relative -- no FP64 needed
__device__ __forceinline__ void dot3t_ff(const float *r, float t, float x, float y, float z,
                                         float &hi, float &lo) {
    const float v[3] = {x, y, z};
    float s = t, c = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p = r[k] * v[k];
        const float pe = fmaf(r[k], v[k], -p);
        const float u = s + p;
        const float bb = u - s;
        const float se = (s - (u - bb)) + (p - bb);
        s = u;
        c += pe + se;
    }
    hi = s + c;
    lo = c - (hi - s);
}

// accurate FP32 (xh + xl) / (zh + zl), rz = 1/zh
__device__ __forceinline__ float ratio_ff(float xh, float xl, float zh, float zl, float rz) {
    const float q0 = xh * rz;
    float e = fmaf(-q0, zh, xh);
    e += xl - q0 * zl;
    return fmaf(e, rz, q0);
}

template <int DEG, bool F16>
__global__ void __launch_bounds__(128)
project_kernel(ViewTable vt, int n, const float *__restrict__ means,
               const float *__restrict__ scales, const float *__restrict__ quats,
               const float *__restrict__ opac, const void *__restrict__ sh_raw, float near_z,
               Filters flt, Record *__restrict__ out) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    float s0 = scales[3 * i], s1 = scales[3 * i + 1], s2 = scales[3 * i + 2];
    const float4 q4 = reinterpret_cast<const float4 *>(quats)[i];
    float op = opac[i];
    // Mip-Splatting's 3D smoothing filter: R S^2 R^T + v I = R (S^2 + v I) R^T,
    // opacity scaled by prod_k s_k / sqrt(s_k^2 + v)
    const float v3 = flt.f3d ? flt.f3d[i] : 0.f;
    // a Gaussian with a non-finite parameter, a zero quaternion or a
    // non-finite colour is culled (empty tile range, in no list)
    bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(s0) && isfinite(s1) &&
                  isfinite(s2) && isfinite(q4.x) && isfinite(q4.y) && isfinite(q4.z) && isfinite(q4.w) &&
                  isfinite(op) && isfinite(v3) &&
                  (q4.x != 0.f || q4.y != 0.f || q4.z != 0.f || q4.w != 0.f);
    if (v3 > 0.f) {
        const float e0 = sqrtf(fmaf(s0, s0, v3)), e1 = sqrtf(fmaf(s1, s1, v3)), e2 = sqrtf(fmaf(s2, s2, v3));
        op *= (s0 / e0) * (s1 / e1) * (s2 / e2);
        s0 = e0;
        s1 = e1;
        s2 = e2;
    }
    // SH coefficient k, channel c (read only for records with tiles: most
    // records are off screen)
    auto sh_coef = [&](int k, int c) -> float {
        if constexpr (F16)
            return __half2float(reinterpret_cast<const __half *>(sh_raw)[(size_t)i * K * 3 + 3 * k + c]);
        else
            return __ldg(reinterpret_cast<const float *>(sh_raw) + (size_t)i * K * 3 + 3 * k + c);
    };
    // M = R(q) S, rows a, columns k: M[a][k] = R[a][k] s_k
    float M[3][3];
    {
        float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
        float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
        float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                         {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                         {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            M[a][0] = R[a][0] * s0;
            M[a][1] = R[a][1] * s1;
            M[a][2] = R[a][2] * s2;
        }
    }
    const double dx = mx, dy = my, dz = mz;
    for (int v = 0; v < vt.n_views; ++v) {
        const ViewDev &V = vt.v[v];
        Record r;
        const double tz = fma((double)V.R[6], dx, fma((double)V.R[7], dy, fma((double)V.R[8], dz, (double)V.t[2])));
        const float zf = __double2float_rn(tz);
        r.a = make_float4(0.f, 0.f, 0.f, 0.f);
        r.b = make_float4(0.f, op, zf, __uint_as_float(kEmptyRange));
        r.c = make_float4(0.f, 0.f, 0.f, __uint_as_float(kEmptyRange));
        if (zf > near_z && finite) {
            float xh, xl, yh, yl, zh, zl;
            dot3t_ff(&V.R[0], V.t[0], mx, my, mz, xh, xl);
            dot3t_ff(&V.R[3], V.t[1], mx, my, mz, yh, yl);
            dot3t_ff(&V.R[6], V.t[2], mx, my, mz, zh, zl);
            const float rz = __frcp_rn(zh);
            const float qx = ratio_ff(xh, xl, zh, zl, rz);
            const float qy = ratio_ff(yh, yl, zh, zl, rz);
            const float u = fmaf(V.fx, qx, V.cx);
            const float w = fmaf(V.fy, qy, V.cy);
            // affine Jacobian with the 1.3 x half-FOV clamp
            const float limx = 1.3f * (0.5f * (float)V.W / V.fx);
            const float limy = 1.3f * (0.5f * (float)V.H / V.fy);
            const float qxc = fminf(limx, fmaxf(-limx, qx));
            const float qyc = fminf(limy, fmaxf(-limy, qy));
            const float J00 = V.fx * rz, J02 = -V.fx * qxc * rz;
            const float J11 = V.fy * rz, J12 = -V.fy * qyc * rz;
            float T0[3], T1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T0[k] = fmaf(J00, V.R[k], J02 * V.R[6 + k]);
                T1[k] = fmaf(J11, V.R[3 + k], J12 * V.R[6 + k]);
            }
            float V0[3], V1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                V0[k] = T0[0] * M[0][k] + T0[1] * M[1][k] + T0[2] * M[2][k];
                V1[k] = T1[0] * M[0][k] + T1[1] * M[1][k] + T1[2] * M[2][k];
            }
            const float A = V0[0] * V0[0] + V0[1] * V0[1] + V0[2] * V0[2];
            const float C = V1[0] * V1[0] + V1[1] * V1[1] + V1[2] * V1[2];
            const float B = dot3_c(V0, V1);
            const float cx_ = diff_prod(V0[1], V1[2], V0[2], V1[1]);
            const float cy_ = diff_prod(V0[2], V1[0], V0[0], V1[2]);
            const float cz_ = diff_prod(V0[0], V1[1], V0[1], V1[0]);
            const float h = flt.kernel;
            const float a = A + h, c = C + h;
            const float det0 = cx_ * cx_ + cy_ * cy_ + cz_ * cz_;      // det(Sigma2D), Lagrange's identity
            const float det = det0 + h * (A + C) + h * h;
            const float rd = 1.0f / det;
            // 2D Mip filter: opacity x sqrt(det Sigma2D / det(Sigma2D + h I))
            const float opv = flt.antialias ? op * sqrtf(det0 * rd) : op;
            // 3-sigma rectangle (inflated by 1e-4 relative + 1e-3 px: a superset)
            const float hx = 3.0f * sqrtf(a) * 1.0001f + 1e-3f;
            const float hy = 3.0f * sqrtf(c) * 1.0001f + 1e-3f;
            // pixel x has centre x+1/2: covered x in [ceil(u-hx-1/2), floor(u+hx-1/2)]
            const float fx0 = ceilf(u - hx - 0.5f), fx1 = floorf(u + hx - 0.5f);
            const float fy0 = ceilf(w - hy - 0.5f), fy1 = floorf(w + hy - 0.5f);
            uint32_t xr = kEmptyRange, yr = kEmptyRange;
            if (fx1 >= 0.f && fx0 <= (float)(V.W - 1) && fy1 >= 0.f && fy0 <= (float)(V.H - 1)) {
                int px0 = (int)fmaxf(fx0, 0.f), px1 = (int)fminf(fx1, (float)(V.W - 1));
                int py0 = (int)fmaxf(fy0, 0.f), py1 = (int)fminf(fy1, (float)(V.H - 1));
                if (px0 <= px1 && py0 <= py1) {
                    xr = pack_range(px0 / vt.tile_w, px1 / vt.tile_w);
                    yr = pack_range(py0 / vt.tile_h, py1 / vt.tile_h);
                }
            }
            // view-dependent colour: SH at the unit direction camera centre ->
            // mean, for a record with tiles (no list holds the others)
            float col[3] = {0.f, 0.f, 0.f};
            if (xr != kEmptyRange) {
                float d0 = mx - V.campos[0], d1 = my - V.campos[1], d2 = mz - V.campos[2];
                float dn = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                d0 *= dn; d1 *= dn; d2 *= dn;
                float Y[K];
                sh_basis<DEG>(d0, d1, d2, Y);
                bool col_ok = true;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float acc = 0.5f;
#pragma unroll
                    for (int k = 0; k < K; ++k) acc = fmaf(Y[k], sh_coef(k, ch), acc);
                    col_ok = col_ok && isfinite(acc);
                    col[ch] = fmaxf(acc, 0.f);
                }
                if (!col_ok) xr = yr = kEmptyRange;
            }
            // conic (c, -B, a) / det, pre-multiplied by K (and 2K for xy)
            r.a = make_float4(u, w, __fmul_rn(kConicScale, c * rd), __fmul_rn(2.f * kConicScale, -B * rd));
            r.b = make_float4(__fmul_rn(kConicScale, a * rd), opv, zf, __uint_as_float(xr));
            r.c = make_float4(col[0], col[1], col[2], __uint_as_float(yr));
        }
        Record *o = out + (size_t)v * n + i;
        o->a = r.a;
        o->b = r.b;
        o->c = r.c;
    }
}

template <int DEG>
cudaError_t launch_deg(const ViewTable &vt, int n, const float *means, const float *scales,
                       const float *quats, const float *opac, const void *sh, bool f16,
                       float near_z, Filters flt, Record *out, cudaStream_t s) {
    dim3 grid((n + 127) / 128);
    if (f16)
        project_kernel<DEG, true><<<grid, 128, 0, s>>>(vt, n, means, scales, quats, opac, sh, near_z, flt, out);
    else
        project_kernel<DEG, false><<<grid, 128, 0, s>>>(vt, n, means, scales, quats, opac, sh, near_z, flt, out);
    return cudaGetLastError();
}

// Mip-Splatting's 3D filter variance: v = s2 (z / f)^2 at the camera with the
// highest sampling rate f / z among those that see the mean (z > near, the
// projected mean inside [0, W] x [0, H]); 0 if none does
__global__ void __launch_bounds__(256)
mip_filter3d_kernel(ViewTable vt, int n, const float *__restrict__ means, float s2, float near_z,
                    float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    float best = 0.f;                                  // largest f / z so far
    for (int v = 0; v < vt.n_views; ++v) {
        const ViewDev &V = vt.v[v];
        const float z = fmaf(V.R[6], mx, fmaf(V.R[7], my, fmaf(V.R[8], mz, V.t[2])));
        if (!(z > near_z)) continue;
        const float x = fmaf(V.R[0], mx, fmaf(V.R[1], my, fmaf(V.R[2], mz, V.t[0])));
        const float y = fmaf(V.R[3], mx, fmaf(V.R[4], my, fmaf(V.R[5], mz, V.t[1])));
        const float u = fmaf(V.fx, x / z, V.cx), w = fmaf(V.fy, y / z, V.cy);
        if (!(u >= 0.f && u <= (float)V.W && w >= 0.f && w <= (float)V.H)) continue;
        best = fmaxf(best, fmaxf(V.fx, V.fy) / z);
    }
    out[i] = best > 0.f ? s2 / (best * best) : 0.f;
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" hm_status hm_project_gaussians(const hm_camera *cams, int32_t n_views, int32_t n,
                                          const float *means, const float *scales,
                                          const float *quats, const float *opacity,
                                          const float *filter_3d, const void *sh, int32_t sh_degree,
                                          int32_t sh_format, const hm_options *opt, void *records,
                                          void *stream) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt)) return HM_ERR_INVALID_ARG;
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (sh_degree < 0 || sh_degree > 3) return fail(HM_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (sh_format != HM_SH_F32 && sh_format != HM_SH_F16) return fail(HM_ERR_INVALID_ARG, "sh_format");
    if (!(opt->kernel_2d >= 0.f && opt->kernel_2d < 1e6f)) return fail(HM_ERR_INVALID_ARG, "kernel_2d");
    if (n == 0) return HM_OK;
    if (!means || !scales || !quats || !opacity || !sh || !records)
        return fail(HM_ERR_INVALID_ARG, "null pointer");
    if (((uintptr_t)records & 15) || ((uintptr_t)quats & 15))
        return fail(HM_ERR_INVALID_ARG, "records and quats must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const bool f16 = sh_format == HM_SH_F16;
    Record *out = reinterpret_cast<Record *>(records);
    const Filters flt{filter_3d, opt->kernel_2d, opt->antialias ? 1 : 0};
    cudaError_t e;
    switch (sh_degree) {
        case 0: e = launch_deg<0>(vt, n, means, scales, quats, opacity, sh, f16, opt->near_gauss, flt, out, s); break;
        case 1: e = launch_deg<1>(vt, n, means, scales, quats, opacity, sh, f16, opt->near_gauss, flt, out, s); break;
        case 2: e = launch_deg<2>(vt, n, means, scales, quats, opacity, sh, f16, opt->near_gauss, flt, out, s); break;
        default: e = launch_deg<3>(vt, n, means, scales, quats, opacity, sh, f16, opt->near_gauss, flt, out, s); break;
    }
    return cuda_status(e);
}

extern "C" hm_status hm_mip_filter_3d(const hm_camera *cams, int32_t n_views, int32_t n, const float *means,
                                      float s2, float near_z, float *filter_3d, void *stream) {
    hm_options o;
    hm_default_options(&o);
    ViewTable vt;
    if (!build_view_table(cams, n_views, &o, &vt)) return HM_ERR_INVALID_ARG;
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (!(s2 > 0.f) || !(near_z >= 0.f)) return fail(HM_ERR_INVALID_ARG, "s2 must be > 0, near_z >= 0");
    if (n == 0) return HM_OK;
    if (!means || !filter_3d) return fail(HM_ERR_INVALID_ARG, "null pointer");
    mip_filter3d_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(vt, n, means, s2, near_z, filter_3d);
    return cuda_status(cudaGetLastError());
}
