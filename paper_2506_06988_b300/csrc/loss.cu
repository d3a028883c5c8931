// loss.cu -- the joint-optimisation loss of the hybrid representation and
// its gradients, fused per image tile:
//   L = (1 - ls) L1(I, I_h) + ls (1 - SSIM(I, I_h)) + lt L_t          (Eq. 3, Sec. 3.4)
//   L_t = mean over pixel-channels of M_T hit (I - I_m)^2,  M_T = 1 / (1 + e^{-k (T - 1/2)})
// over all pixel-channel elements of all cameras (N of them); SSIM with the
// 11 x 11 Gaussian window (sigma 1.5, separable, zero outside the image),
// C1 = 0.01^2, C2 = 0.03^2.  M_T is a mask (no gradient to T).
//
// Two passes over 16 x 16 tiles, a CTA per (tile, channel):
//  * ssim_fwd: the five window sums (mu_x, mu_y, E[x^2], E[y^2], E[xy]) by
//    a horizontal then a vertical 11-tap pass through shared memory (halo 5),
//    the SSIM map and its partial derivatives with respect to the window
//    sums -- D_mu = dS/dmu_x, D_xx = dS/dE[x^2], D_xy = dS/dE[xy] -- to
//    global scratch; the pointwise L1 and texture-loss terms, dL/dI_m; the
//    three sums (FP64 atomics, one per CTA).
//  * ssim_bwd: since mu_x, E[x^2], E[xy] at pixel p are window sums of x,
//    x^2 and x y, dSSIM_total/dx(q) = (w * D_mu)(q) + 2 x(q) (w * D_xx)(q)
//    + y(q) (w * D_xy)(q): the same separable window over the three maps,
//    then dL/dI_h = ((1 - ls) sign(x - y) - ls dSSIM/dx) / N.
#include "hm_host.h"

namespace hm {

namespace {

constexpr int kLT = 16;              // output tile edge
constexpr int kRad = 5;              // window radius
constexpr int kTaps = 2 * kRad + 1;  // 11
constexpr int kHalo = kLT + 2 * kRad;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Taps {
    float g[kTaps];
};

__device__ __forceinline__ double block_sum(double v, double *s_red) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (t == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += s_red[k];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kLT *kLT)
ssim_fwd_kernel(ViewTable vt, Taps tp, const float *__restrict__ x_all, const float *__restrict__ y_all,
                const float *__restrict__ m_all, const float *__restrict__ T_all,
                const float *__restrict__ md_all, float k_mask, float mesh_grad_scale,
                float *__restrict__ d_mu, float *__restrict__ d_xx, float *__restrict__ d_xy,
                float *__restrict__ dL_dmesh, double *__restrict__ sums) {
    __shared__ float s_x[kHalo][kHalo], s_y[kHalo][kHalo];
    __shared__ float s_h[5][kHalo][kLT];
    __shared__ double s_red[kLT * kLT / 32];
    const int gt = blockIdx.x, ch = blockIdx.y;
    const int v = view_of_tile(vt, gt);
    const ViewDev &V = vt.v[v];
    const int local = gt - V.tile_off;
    const int px0 = (local % V.tiles_x) * kLT, py0 = (local / V.tiles_x) * kLT;
    const long long npx = (long long)V.W * V.H;
    const float *x = x_all + 3 * V.pix_off + ch * npx;
    const float *y = y_all + 3 * V.pix_off + ch * npx;
    const int t = threadIdx.x;
    for (int i = t; i < kHalo * kHalo; i += kLT * kLT) {
        const int r = i / kHalo, c = i % kHalo;
        const int gx = px0 - kRad + c, gy = py0 - kRad + r;
        float xv = 0.f, yv = 0.f;
        if (gx >= 0 && gx < V.W && gy >= 0 && gy < V.H) {
            xv = x[(long long)gy * V.W + gx];
            yv = y[(long long)gy * V.W + gx];
        }
        s_x[r][c] = xv;
        s_y[r][c] = yv;
    }
    __syncthreads();
    for (int i = t; i < kHalo * kLT; i += kLT * kLT) {
        const int r = i / kLT, c = i % kLT;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) {
            const float g = tp.g[k], xv = s_x[r][c + k], yv = s_y[r][c + k];
            a = fmaf(g, xv, a);
            b = fmaf(g, yv, b);
            aa = fmaf(g, xv * xv, aa);
            bb = fmaf(g, yv * yv, bb);
            ab = fmaf(g, xv * yv, ab);
        }
        s_h[0][r][c] = a; s_h[1][r][c] = b; s_h[2][r][c] = aa; s_h[3][r][c] = bb; s_h[4][r][c] = ab;
    }
    __syncthreads();
    const int r = t / kLT, c = t % kLT;
    const int px = px0 + c, py = py0 + r;
    const bool in = px < V.W && py < V.H;
    double ssum = 0.0, l1 = 0.0, lt = 0.0;
    if (in) {
        float mx = 0.f, my = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) {
            const float g = tp.g[k];
            mx = fmaf(g, s_h[0][r + k][c], mx);
            my = fmaf(g, s_h[1][r + k][c], my);
            sxx = fmaf(g, s_h[2][r + k][c], sxx);
            syy = fmaf(g, s_h[3][r + k][c], syy);
            sxy = fmaf(g, s_h[4][r + k][c], sxy);
        }
        const float vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
        const float A1 = fmaf(2.f * mx, my, kC1), A2 = fmaf(2.f, cxy, kC2);
        const float B1 = fmaf(mx, mx, fmaf(my, my, kC1)), B2 = vx + vy + kC2;
        const float S = (A1 * A2) / (B1 * B2);
        // dS/d(mu_x, E[x^2], E[xy]) with sigma_x^2 = E[x^2] - mu_x^2 and
        // sigma_xy = E[xy] - mu_x mu_y
        const long long lp = (long long)py * V.W + px;
        const long long o = 3 * V.pix_off + ch * npx + lp;
        d_mu[o] = S * (2.f * my / A1 - 2.f * my / A2 - 2.f * mx / B1 + 2.f * mx / B2);
        d_xx[o] = -S / B2;
        d_xy[o] = 2.f * S / A2;
        ssum = S;
        const float xv = s_x[r + kRad][c + kRad], yv = s_y[r + kRad][c + kRad];
        l1 = fabsf(xv - yv);
        if (m_all) {
            const float *m = m_all + 3 * V.pix_off + ch * npx;
            const bool hit = md_all[V.pix_off + lp] < INFINITY;
            float g = 0.f;
            if (hit) {
                const float mt = 1.f / (1.f + expf(-k_mask * (T_all[V.pix_off + lp] - 0.5f)));
                const float d = yv - m[lp];
                lt = (double)(mt * d * d);
                g = mesh_grad_scale * mt * -d;     // d/dm of mt (y - m)^2, times lt / N
            }
            dL_dmesh[o] = g;
        }
    }
    ssum = block_sum(ssum, s_red);
    l1 = block_sum(l1, s_red);
    lt = block_sum(lt, s_red);
    if (t == 0) {
        atomicAdd(&sums[0], l1);
        atomicAdd(&sums[1], ssum);
        atomicAdd(&sums[2], lt);
    }
}

__global__ void __launch_bounds__(kLT *kLT)
ssim_bwd_kernel(ViewTable vt, Taps tp, const float *__restrict__ x_all, const float *__restrict__ y_all,
                const float *__restrict__ d_mu, const float *__restrict__ d_xx, const float *__restrict__ d_xy,
                float l1_scale, float ssim_scale, float *__restrict__ dL_drgb) {
    __shared__ float s_d[3][kHalo][kHalo];
    __shared__ float s_h[3][kHalo][kLT];
    const int gt = blockIdx.x, ch = blockIdx.y;
    const int v = view_of_tile(vt, gt);
    const ViewDev &V = vt.v[v];
    const int local = gt - V.tile_off;
    const int px0 = (local % V.tiles_x) * kLT, py0 = (local / V.tiles_x) * kLT;
    const long long npx = (long long)V.W * V.H;
    const long long base = 3 * V.pix_off + ch * npx;
    const int t = threadIdx.x;
    for (int i = t; i < kHalo * kHalo; i += kLT * kLT) {
        const int r = i / kHalo, c = i % kHalo;
        const int gx = px0 - kRad + c, gy = py0 - kRad + r;
        float a = 0.f, b = 0.f, e = 0.f;
        if (gx >= 0 && gx < V.W && gy >= 0 && gy < V.H) {
            const long long o = base + (long long)gy * V.W + gx;
            a = d_mu[o];
            b = d_xx[o];
            e = d_xy[o];
        }
        s_d[0][r][c] = a;
        s_d[1][r][c] = b;
        s_d[2][r][c] = e;
    }
    __syncthreads();
    for (int i = t; i < kHalo * kLT; i += kLT * kLT) {
        const int r = i / kLT, c = i % kLT;
        float a = 0.f, b = 0.f, e = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) {
            const float g = tp.g[k];
            a = fmaf(g, s_d[0][r][c + k], a);
            b = fmaf(g, s_d[1][r][c + k], b);
            e = fmaf(g, s_d[2][r][c + k], e);
        }
        s_h[0][r][c] = a; s_h[1][r][c] = b; s_h[2][r][c] = e;
    }
    __syncthreads();
    const int r = t / kLT, c = t % kLT;
    const int px = px0 + c, py = py0 + r;
    if (px >= V.W || py >= V.H) return;
    float a = 0.f, b = 0.f, e = 0.f;
#pragma unroll
    for (int k = 0; k < kTaps; ++k) {
        const float g = tp.g[k];
        a = fmaf(g, s_h[0][r + k][c], a);
        b = fmaf(g, s_h[1][r + k][c], b);
        e = fmaf(g, s_h[2][r + k][c], e);
    }
    const long long o = base + (long long)py * V.W + px;
    const float xv = x_all[o], yv = y_all[o];
    const float dS = fmaf(2.f * xv, b, fmaf(yv, e, a));
    const float sg = xv > yv ? 1.f : (xv < yv ? -1.f : 0.f);
    dL_drgb[o] = fmaf(l1_scale, sg, -ssim_scale * dS);
}

__global__ void loss_final_kernel(const double *sums, double inv_n, double ls, double lt, double *out) {
    const double l1 = sums[0] * inv_n, ss = sums[1] * inv_n, t = sums[2] * inv_n;
    out[0] = l1;
    out[1] = ss;
    out[2] = t;
    out[3] = (1.0 - ls) * l1 + ls * (1.0 - ss) + lt * t;
}

bool loss_view_table(const hm_camera *cams, int32_t n_views, ViewTable *vt) {
    hm_options o;
    hm_default_options(&o);
    o.tile_w = o.tile_h = kLT;
    return build_view_table(cams, n_views, &o, vt);
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" void hm_default_loss_params(hm_loss_params *p) {
    if (!p) return;
    p->lambda_ssim = 0.2f;
    p->lambda_t = 0.1f;
    p->k = 20.0f;
}

extern "C" size_t hm_hybrid_loss_workspace_size(const hm_camera *cams, int32_t n_views) {
    ViewTable vt;
    if (!loss_view_table(cams, n_views, &vt)) return 0;
    return sizeof(float) * 9 * (size_t)vt.total_pixels + 3 * 256 + 256;
}

extern "C" hm_status hm_hybrid_loss(const hm_camera *cams, int32_t n_views, const float *out_rgb,
                                    const float *target, const float *mesh_rgb, const float *out_T,
                                    const float *mesh_depth, const hm_loss_params *p,
                                    double *loss_out, float *dL_drgb, float *dL_dmesh, void *ws,
                                    size_t ws_bytes, void *stream) {
    ViewTable vt;
    if (!loss_view_table(cams, n_views, &vt)) return HM_ERR_INVALID_ARG;
    if (!p || !out_rgb || !target || !loss_out || !dL_drgb) return fail(HM_ERR_INVALID_ARG, "null pointer");
    const bool mesh = mesh_rgb != nullptr;
    if (mesh && (!out_T || !mesh_depth || !dL_dmesh))
        return fail(HM_ERR_INVALID_ARG, "the texture loss needs mesh_rgb, out_T, mesh_depth and dL_dmesh");
    if (!(p->lambda_ssim >= 0.f && p->lambda_ssim <= 1.f) || !(p->lambda_t >= 0.f))
        return fail(HM_ERR_INVALID_ARG, "loss weights out of range");
    const size_t need = hm_hybrid_loss_workspace_size(cams, n_views);
    if (!ws || ws_bytes < need) return fail(HM_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    WsCarver c(ws);
    const size_t np3 = 3 * (size_t)vt.total_pixels;
    float *d_mu = c.take<float>(np3), *d_xx = c.take<float>(np3), *d_xy = c.take<float>(np3);
    double *sums = c.take<double>(3);
    cudaError_t e = cudaMemsetAsync(sums, 0, 3 * sizeof(double), s);
    if (e != cudaSuccess) return cuda_status(e);
    Taps tp;
    {
        double g[kTaps], tot = 0.0;
        for (int k = 0; k < kTaps; ++k) {
            const double d = k - kRad;
            g[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
            tot += g[k];
        }
        for (int k = 0; k < kTaps; ++k) tp.g[k] = (float)(g[k] / tot);
    }
    const double n_el = (double)np3;
    dim3 grid(vt.total_tiles, 3);
    ssim_fwd_kernel<<<grid, kLT * kLT, 0, s>>>(vt, tp, out_rgb, target, mesh ? mesh_rgb : nullptr, out_T,
                                               mesh_depth, p->k, (float)(2.0 * p->lambda_t / n_el), d_mu, d_xx,
                                               d_xy, dL_dmesh, sums);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    ssim_bwd_kernel<<<grid, kLT * kLT, 0, s>>>(vt, tp, out_rgb, target, d_mu, d_xx, d_xy,
                                               (float)((1.0 - p->lambda_ssim) / n_el),
                                               (float)(p->lambda_ssim / n_el), dL_drgb);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    loss_final_kernel<<<1, 1, 0, s>>>(sums, 1.0 / n_el, p->lambda_ssim, p->lambda_t, loss_out);
    return cuda_status(cudaGetLastError());
}
