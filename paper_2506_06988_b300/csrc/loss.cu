// loss.cu -- the joint-optimisation loss of the hybrid representation and
// its gradients, fused per image tile:
//   L = (1 - ls) L1(I, I_h) + ls (1 - SSIM(I, I_h)) + lt L_t          (Eq. 3, Eq. 7)
//   L_t = mean over pixel-channels of M_T hit (I - I_m)^2              (Eq. 5)
//   M_T = 1 / (1 + e^{-k (T - 1/2)})                                   (Eq. 6)
// over all pixel-channel elements of all cameras (N of them); SSIM with the
// 11 x 11 Gaussian window (sigma 1.5, separable, zero outside the image),
// C1 = 0.01^2, C2 = 0.03^2.  M_T is a mask (no gradient to T).
//
// Two passes over 32 x 32 tiles, a CTA of 256 threads per (tile, channel):
//  * ssim_fwd: the five window sums (mu_x, mu_y, E[x^2], E[y^2], E[xy]) by
//    a horizontal then a vertical 11-tap pass through shared memory (halo 5,
//    (x, y) interleaved; each thread computes 4 adjacent outputs of a pass
//    from 14 loaded values; both passes carry the (x, y) pairs in FP32x2
//    FMAs; all halo loads are issued before the first shared store),
//    the SSIM map and its partial derivatives with respect to the window
//    sums -- D_mu = dS/dmu_x, D_xx = dS/dE[x^2], D_xy = dS/dE[xy] -- to
//    global scratch ((D_mu, D_xx) interleaved, D_xy a plane of its own); the pointwise L1 and texture-loss terms, dL/dI_m; the
//    CTA's three partial sums (FP32 within a warp, FP64 across warps) to
//    its own slot.  The SSIM quotient uses the hardware's approximate
//    reciprocal (relative error ~2^-23).
//  * ssim_bwd: since mu_x, E[x^2], E[xy] at pixel p are window sums of x,
//    x^2 and x y, dSSIM_total/dx(q) = (w * D_mu)(q) + 2 x(q) (w * D_xx)(q)
//    + y(q) (w * D_xy)(q): the same separable window over the three maps,
//    then dL/dI_h = ((1 - ls) sign(x - y) - ls dSSIM/dx) / N.
//  * loss_reduce / loss_final: the partial sums in a fixed order over a
//    fixed partition (the loss is bitwise reproducible) and the weighted
//    total.
#include "hm_host.h"

namespace hm {

namespace {

constexpr int kLT = 32;              // output tile edge
constexpr int kNT = 256;             // threads per CTA
constexpr int kRad = 5;              // window radius
constexpr int kTaps = 2 * kRad + 1;  // 11
constexpr int kHalo = kLT + 2 * kRad;   // 42 rows / columns with the halo
constexpr int kHS = 48;              // float halo row stride (float4-aligned, >= 4*7 + 16; 192 B)
constexpr int kHS2 = 50;             // float2 halo row stride (400 B: rows r, r+1 16 B apart mod 128)
// The horizontal pass gives the eight threads of a shared-memory phase two
// adjacent rows and four column groups each (see horiz_item), so with these
// strides their 16-byte accesses fall in distinct bank groups.  The pass's
// outputs have unpadded rows; odd rows are stored with their columns
// swizzled (float2 maps: column ^ 2, float maps: column ^ 16), which does the
// same for the stores, and the vertical pass reads them back through the
// same swizzle.
__device__ __forceinline__ void horiz_item(int i, int &r, int &c0) {
    r = 2 * (i >> 4) + ((i >> 2) & 1);
    c0 = 4 * ((i & 3) | (((i >> 3) & 1) << 2));
}
constexpr int kOut = 4;              // outputs per thread per pass
constexpr int kSpan = kOut + kTaps - 1;   // 14 inputs per 4 outputs
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Taps {
    float g[kTaps];
};

constexpr int kHaloSlots = (kHalo * kHalo + kNT - 1) / kNT;   // 7 halo elements per thread

// halo element s of this thread: row r, column c; false past the halo
__device__ __forceinline__ bool halo_slot(int s, int &r, int &c) {
    const int i = threadIdx.x + s * kNT;
    r = i / kHalo;
    c = i - r * kHalo;
    return i < kHalo * kHalo;
}

__device__ __forceinline__ void load_span2(const float2 *row, float2 (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 f = *reinterpret_cast<const float4 *>(row + 2 * q);
        v[2 * q] = make_float2(f.x, f.y);
        v[2 * q + 1] = make_float2(f.z, f.w);
    }
}

// out[o] = sum_k g[k] v[o + k] on both lanes of a pair, o < 4
__device__ __forceinline__ void taps4x2(const Taps &tp, const float2 *v, float2 (&out)[kOut]) {
#pragma unroll
    for (int o = 0; o < kOut; ++o) out[o] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kTaps; ++k)
#pragma unroll
        for (int o = 0; o < kOut; ++o) out[o] = __ffma2_rn(make_float2(tp.g[k], tp.g[k]), v[o + k], out[o]);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void load_span(const float *row, float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 f = *reinterpret_cast<const float4 *>(row + 4 * q);
        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
    }
}

// out[o] = sum_k g[k] v[o + k], o < 4
__device__ __forceinline__ void taps4(const Taps &tp, const float *v, float (&out)[kOut]) {
#pragma unroll
    for (int o = 0; o < kOut; ++o) out[o] = 0.f;
#pragma unroll
    for (int k = 0; k < kTaps; ++k)
#pragma unroll
        for (int o = 0; o < kOut; ++o) out[o] = fmaf(tp.g[k], v[o + k], out[o]);
}

// vertical pass, thread (column c, rows 4 rg .. 4 rg + 3): each loaded row
// value feeds the (up to 4) outputs whose window covers it; odd rows are
// read through the column swizzle (rows 4 rg + j have the parity of j)
__device__ __forceinline__ void vert4x2(const Taps &tp, const float2 (*sh)[kLT], int c, int rg,
                                        float2 (&out)[kOut]) {
#pragma unroll
    for (int o = 0; o < kOut; ++o) out[o] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kSpan; ++j) {
        const float2 v = sh[kOut * rg + j][(j & 1) ? (c ^ 2) : c];
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            const int k = j - o;
            if (k >= 0 && k < kTaps) out[o] = __ffma2_rn(make_float2(tp.g[k], tp.g[k]), v, out[o]);
        }
    }
}

__device__ __forceinline__ void vert4x1(const Taps &tp, const float (*sh)[kLT], int c, int rg, float (&out)[kOut]) {
#pragma unroll
    for (int o = 0; o < kOut; ++o) out[o] = 0.f;
#pragma unroll
    for (int j = 0; j < kSpan; ++j) {
        const float v = sh[kOut * rg + j][(j & 1) ? (c ^ 16) : c];
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            const int k = j - o;
            if (k >= 0 && k < kTaps) out[o] = fmaf(tp.g[k], v, out[o]);
        }
    }
}

// FP32 warp sums (each lane holds a few pixels), then the eight warp sums in
// FP64 in a fixed order; the result lands in s_red[q][0]
__device__ __forceinline__ void block_sum3_warps(float (&v)[3], double (*s_red)[kNT / 32]) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) s_red[q][w] = (double)v[q];
    }
    __syncthreads();
    if (t < 3) {
        double r = 0.0;
        for (int k = 0; k < kNT / 32; ++k) r += s_red[t][k];
        s_red[t][0] = r;
    }
    __syncthreads();
}

__device__ __forceinline__ void block_sum3(double (&v)[3], double (*s_red)[kNT / 32]) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) s_red[q][w] = v[q];
    }
    __syncthreads();
    if (t < 3) {
        double r = 0.0;
        for (int k = 0; k < kNT / 32; ++k) r += s_red[t][k];
        s_red[t][0] = r;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = s_red[q][0];
}

// Target intensity at element o: FP32 values, or 8-bit codes read as
// code / 255 (correctly rounded, as hm_decode_u8 writes them: a 256-entry
// table each CTA fills in shared memory), so a loss on the codes equals the
// loss on their decoded image bit for bit.
template <typename TT>
struct Target {
    const TT *y;
    float *lut;      // 8-bit codes: the CTA's table
    // fills the table (called by the whole CTA; ends with a barrier)
    __device__ __forceinline__ void init() {
        if constexpr (sizeof(TT) == 1) {
            for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = __fdiv_rn((float)i, 255.f);
            __syncthreads();
        }
    }
    __device__ __forceinline__ float operator()(long long o) const {
        if constexpr (sizeof(TT) == 1) return lut[y[o]];
        else return y[o];
    }
};

template <typename TT>
__global__ void __launch_bounds__(kNT, 5)
ssim_fwd_kernel(ViewTable vt, Taps tp, const float *__restrict__ x_all, const TT *__restrict__ y_all,
                const float *__restrict__ m_all, const float *__restrict__ T_all,
                const float *__restrict__ md_all, float k_mask, float mesh_grad_scale,
                float2 *__restrict__ d_mu_xx, float *__restrict__ d_xy,
                float *__restrict__ dL_dmesh, double *__restrict__ partials) {
    __shared__ __align__(16) float2 s_in[kHalo][kHS2];  // (x, y) interleaved
    __shared__ __align__(16) float2 s_m[kHalo][kLT];    // (w*x, w*y) along rows
    __shared__ __align__(16) float2 s_q[kHalo][kLT];    // (w*x^2, w*y^2)
    __shared__ __align__(16) float s_c[kHalo][kLT];     // w*(x y)
    __shared__ double s_red[3][kNT / 32];
    const int gt = blockIdx.x, ch = blockIdx.y;
    const int v = view_of_tile(vt, gt);
    const ViewDev &V = vt.v[v];
    const int local = gt - V.tile_off;
    const int px0 = (local % V.tiles_x) * kLT, py0 = (local / V.tiles_x) * kLT;
    const long long npx = (long long)V.W * V.H;
    const long long base = 3 * V.pix_off + ch * npx;
    __shared__ float s_lut[256];
    Target<TT> tgt{y_all + base, s_lut};
    tgt.init();
    const int t = threadIdx.x;
    {
        // every load of the halo issued before the first shared-memory store
        const float *x = x_all + base;
        const int W = V.W, H = V.H;
        float2 hv[kHaloSlots];
#pragma unroll
        for (int k = 0; k < kHaloSlots; ++k) {
            int r, c;
            const bool in = halo_slot(k, r, c);
            const int gx = px0 - kRad + c, gy = py0 - kRad + r;
            hv[k] = make_float2(0.f, 0.f);
            if (in && gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const long long o = (long long)gy * W + gx;
                hv[k] = make_float2(x[o], tgt(o));
            }
        }
#pragma unroll
        for (int k = 0; k < kHaloSlots; ++k) {
            int r, c;
            if (halo_slot(k, r, c)) s_in[r][c] = hv[k];
        }
    }
    __syncthreads();
    // horizontal: (row r, columns c0 .. c0 + 3) of the five products, the
    // (x, y) pairs in FP32x2
    for (int i = t; i < kHalo * (kLT / kOut); i += kNT) {
        int r, c0;
        horiz_item(i, r, c0);
        float2 xy[16], sq[kSpan], mm[kOut], qq[kOut];
        float pr[kSpan], o[kOut];
        load_span2(&s_in[r][c0], xy);
#pragma unroll
        for (int j = 0; j < kSpan; ++j) {
            sq[j] = __fmul2_rn(xy[j], xy[j]);
            pr[j] = xy[j].x * xy[j].y;
        }
        taps4x2(tp, xy, mm);
        taps4x2(tp, sq, qq);
        taps4(tp, pr, o);
        const int sw2 = (r & 1) * 2, sw1 = (r & 1) * 16;     // odd rows: swizzled columns
        *reinterpret_cast<float4 *>(&s_m[r][c0 ^ sw2]) = make_float4(mm[0].x, mm[0].y, mm[1].x, mm[1].y);
        *reinterpret_cast<float4 *>(&s_m[r][(c0 + 2) ^ sw2]) = make_float4(mm[2].x, mm[2].y, mm[3].x, mm[3].y);
        *reinterpret_cast<float4 *>(&s_q[r][c0 ^ sw2]) = make_float4(qq[0].x, qq[0].y, qq[1].x, qq[1].y);
        *reinterpret_cast<float4 *>(&s_q[r][(c0 + 2) ^ sw2]) = make_float4(qq[2].x, qq[2].y, qq[3].x, qq[3].y);
        *reinterpret_cast<float4 *>(&s_c[r][c0 ^ sw1]) = make_float4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();
    const int c = t & 31, rg = t >> 5;
    float2 mu[kOut], ex2[kOut];
    float exy[kOut];
    vert4x2(tp, s_m, c, rg, mu);
    vert4x2(tp, s_q, c, rg, ex2);
    vert4x1(tp, s_c, c, rg, exy);
    const int px = px0 + c;
    float ssum = 0.f, l1 = 0.f, lt = 0.f;
#pragma unroll
    for (int q = 0; q < kOut; ++q) {
        const int r = kOut * rg + q, py = py0 + r;
        if (px >= V.W || py >= V.H) continue;
        const float mx = mu[q].x, my = mu[q].y;
        const float vx = ex2[q].x - mx * mx, vy = ex2[q].y - my * my, cxy = exy[q] - mx * my;
        const float A1 = fmaf(2.f * mx, my, kC1), A2 = fmaf(2.f, cxy, kC2);
        const float B1 = fmaf(mx, mx, fmaf(my, my, kC1)), B2 = vx + vy + kC2;
        const float rA1 = rcp_approx(A1), rA2 = rcp_approx(A2), rB1 = rcp_approx(B1), rB2 = rcp_approx(B2);
        const float S = (A1 * A2) * (rB1 * rB2);
        // dS/d(mu_x, E[x^2], E[xy]) with sigma_x^2 = E[x^2] - mu_x^2 and
        // sigma_xy = E[xy] - mu_x mu_y
        const long long lp = (long long)py * V.W + px;
        const long long o = base + lp;
        const float dmu = 2.f * S * fmaf(my, rA1 - rA2, mx * (rB2 - rB1));
        d_mu_xx[o] = make_float2(dmu, -S * rB2);
        d_xy[o] = 2.f * S * rA2;
        ssum += S;
        const float2 xyc = s_in[r + kRad][c + kRad];
        const float xv = xyc.x, yv = xyc.y;
        l1 += fabsf(xv - yv);
        if (m_all) {
            const bool hit = md_all[V.pix_off + lp] < INFINITY;
            float g = 0.f;
            if (hit) {
                const float mt = 1.f / (1.f + expf(-k_mask * (T_all[V.pix_off + lp] - 0.5f)));
                const float d = yv - m_all[o];
                lt = fmaf(mt * d, d, lt);
                g = mesh_grad_scale * mt * -d;     // d/dm of mt (y - m)^2, times lt / N
            }
            dL_dmesh[o] = g;
        }
    }
    float sums[3] = {l1, ssum, lt};
    block_sum3_warps(sums, s_red);
    if (t < 3) partials[3 * ((long long)ch * gridDim.x + gt) + t] = s_red[t][0];
}

template <typename TT>
__global__ void __launch_bounds__(kNT)
ssim_bwd_kernel(ViewTable vt, Taps tp, const float *__restrict__ x_all, const TT *__restrict__ y_all,
                const float2 *__restrict__ d_mu_xx, const float *__restrict__ d_xy,
                float l1_scale, float ssim_scale, float *__restrict__ dL_drgb) {
    __shared__ __align__(16) float2 s_d[kHalo][kHS2];   // (D_mu, D_xx) interleaved
    __shared__ __align__(16) float s_dxy[kHalo][kHS];   // D_xy
    __shared__ __align__(16) float2 s_ab[kHalo][kLT];   // w*D_mu, w*D_xx along rows
    __shared__ __align__(16) float s_e[kHalo][kLT];     // w*D_xy
    const int gt = blockIdx.x, ch = blockIdx.y;
    const int v = view_of_tile(vt, gt);
    const ViewDev &V = vt.v[v];
    const int local = gt - V.tile_off;
    const int px0 = (local % V.tiles_x) * kLT, py0 = (local / V.tiles_x) * kLT;
    const long long npx = (long long)V.W * V.H;
    const long long base = 3 * V.pix_off + ch * npx;
    const int t = threadIdx.x;
    __shared__ float s_lut[256];
    Target<TT> tgt{y_all, s_lut};
    tgt.init();
    // this thread's four output pixels: x and y fetched now, used at the end
    float xo[kOut], yo[kOut];
#pragma unroll
    for (int q = 0; q < kOut; ++q) {
        const int px = px0 + (t & 31), py = py0 + kOut * (t >> 5) + q;
        xo[q] = yo[q] = 0.f;
        if (px < V.W && py < V.H) {
            const long long o = base + (long long)py * V.W + px;
            xo[q] = x_all[o];
            yo[q] = tgt(o);
        }
    }
    {
        const float2 *ab = d_mu_xx + base;
        const float *e = d_xy + base;
        const int W = V.W, H = V.H;
        float2 ha[kHaloSlots];
        float he[kHaloSlots];
#pragma unroll
        for (int k = 0; k < kHaloSlots; ++k) {
            int r, c;
            const bool in = halo_slot(k, r, c);
            const int gx = px0 - kRad + c, gy = py0 - kRad + r;
            ha[k] = make_float2(0.f, 0.f);
            he[k] = 0.f;
            if (in && gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const long long o = (long long)gy * W + gx;
                ha[k] = ab[o];
                he[k] = e[o];
            }
        }
#pragma unroll
        for (int k = 0; k < kHaloSlots; ++k) {
            int r, c;
            if (halo_slot(k, r, c)) {
                s_d[r][c] = ha[k];
                s_dxy[r][c] = he[k];
            }
        }
    }
    __syncthreads();
    for (int i = t; i < kHalo * (kLT / kOut); i += kNT) {
        int r, c0;
        horiz_item(i, r, c0);
        const int sw2 = (r & 1) * 2, sw1 = (r & 1) * 16;     // odd rows: swizzled columns
        float2 dv[16], oab[kOut];
        load_span2(&s_d[r][c0], dv);
        taps4x2(tp, dv, oab);
        *reinterpret_cast<float4 *>(&s_ab[r][c0 ^ sw2]) = make_float4(oab[0].x, oab[0].y, oab[1].x, oab[1].y);
        *reinterpret_cast<float4 *>(&s_ab[r][(c0 + 2) ^ sw2]) = make_float4(oab[2].x, oab[2].y, oab[3].x, oab[3].y);
        float vs[16], o[kOut];
        load_span(&s_dxy[r][c0], vs);
        taps4(tp, vs, o);
        *reinterpret_cast<float4 *>(&s_e[r][c0 ^ sw1]) = make_float4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();
    const int c = t & 31, rg = t >> 5;
    float2 ab[kOut];
    float e[kOut];
    vert4x2(tp, s_ab, c, rg, ab);
    vert4x1(tp, s_e, c, rg, e);
    const int px = px0 + c;
#pragma unroll
    for (int q = 0; q < kOut; ++q) {
        const int py = py0 + kOut * rg + q;
        if (px >= V.W || py >= V.H) continue;
        const long long o = base + (long long)py * V.W + px;
        const float xv = xo[q], yv = yo[q];
        const float dS = fmaf(2.f * xv, ab[q].y, fmaf(yv, e[q], ab[q].x));
        const float sg = xv > yv ? 1.f : (xv < yv ? -1.f : 0.f);
        dL_drgb[o] = fmaf(l1_scale, sg, -ssim_scale * dS);
    }
}

// The loss without its SSIM term (lambda_ssim == 0): pointwise, a thread per
// pixel of all cameras over its three channels -- L1 and its gradient
// sign(x - y) / N, and the texture loss as in the tiled pass; per-CTA
// partial sums for the fixed-order final reduction (the SSIM slot is 0).
template <typename TT>
__global__ void __launch_bounds__(kNT)
l1_loss_kernel(ViewTable vt, const float *__restrict__ x_all, const TT *__restrict__ y_all,
               const float *__restrict__ m_all, const float *__restrict__ T_all, const float *__restrict__ md_all,
               float k_mask, float l1_scale, float mesh_grad_scale, float *__restrict__ dL_drgb,
               float *__restrict__ dL_dmesh, double *__restrict__ partials) {
    __shared__ double s_red[3][kNT / 32];
    __shared__ float s_lut[256];
    Target<TT> tgt{y_all, s_lut};
    tgt.init();
    float l1 = 0.f, lt = 0.f;
    for (long long gp = (long long)blockIdx.x * kNT + threadIdx.x; gp < vt.total_pixels;
         gp += (long long)gridDim.x * kNT) {
        const int v = view_of_pixel(vt, gp);
        const ViewDev &V = vt.v[v];
        const long long lp = gp - V.pix_off, npx = (long long)V.W * V.H;
        float mt = 0.f;
        const bool hit = m_all && md_all[gp] < INFINITY;
        if (hit) mt = 1.f / (1.f + expf(-k_mask * (T_all[gp] - 0.5f)));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long o = 3 * V.pix_off + c * npx + lp;
            const float xv = x_all[o], yv = tgt(o);
            l1 += fabsf(xv - yv);
            dL_drgb[o] = xv > yv ? l1_scale : (xv < yv ? -l1_scale : 0.f);
            if (m_all) {
                float g = 0.f;
                if (hit) {
                    const float d = yv - m_all[o];
                    lt = fmaf(mt * d, d, lt);
                    g = mesh_grad_scale * mt * -d;
                }
                dL_dmesh[o] = g;
            }
        }
    }
    double sums[3] = {(double)l1, 0.0, (double)lt};
    block_sum3(sums, s_red);
    if (threadIdx.x < 3) partials[3 * (long long)blockIdx.x + threadIdx.x] = s_red[threadIdx.x][0];
}

// The same pointwise pass four pixels at a time (16-byte loads and stores of
// each plane, one 4-byte load of 8-bit codes) when every camera's pixel count
// is a multiple of 4 and the buffers are 16-byte aligned: the same per-element
// arithmetic, so the gradients are those of l1_loss_kernel bit for bit.
template <typename TT>
__global__ void __launch_bounds__(kNT)
l1_loss4_kernel(ViewTable vt, const float *__restrict__ x_all, const TT *__restrict__ y_all,
                const float *__restrict__ m_all, const float *__restrict__ T_all, const float *__restrict__ md_all,
                float k_mask, float l1_scale, float mesh_grad_scale, float *__restrict__ dL_drgb,
                float *__restrict__ dL_dmesh, double *__restrict__ partials) {
    __shared__ double s_red[3][kNT / 32];
    __shared__ float s_lut[256];
    Target<TT> tgt{y_all, s_lut};
    tgt.init();
    float l1 = 0.f, lt = 0.f;
    const long long nq = vt.total_pixels / 4;
    for (long long qd = (long long)blockIdx.x * kNT + threadIdx.x; qd < nq; qd += (long long)gridDim.x * kNT) {
        const long long gp = 4 * qd;
        const int v = view_of_pixel(vt, gp);
        const ViewDev &V = vt.v[v];
        const long long lp = gp - V.pix_off, npx = (long long)V.W * V.H;
        float mt[4] = {0.f, 0.f, 0.f, 0.f};
        bool hit[4] = {false, false, false, false};
        if (m_all) {
            const float4 md = *reinterpret_cast<const float4 *>(md_all + gp);
            const float4 T4 = *reinterpret_cast<const float4 *>(T_all + gp);
            const float mdv[4] = {md.x, md.y, md.z, md.w}, Tv[4] = {T4.x, T4.y, T4.z, T4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                hit[u] = mdv[u] < INFINITY;
                if (hit[u]) mt[u] = 1.f / (1.f + expf(-k_mask * (Tv[u] - 0.5f)));
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long o = 3 * V.pix_off + c * npx + lp;
            const float4 x4 = *reinterpret_cast<const float4 *>(x_all + o);
            const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
            float yv[4];
            if constexpr (sizeof(TT) == 1) {
                const uint32_t w = *reinterpret_cast<const uint32_t *>(y_all + o);
#pragma unroll
                for (int u = 0; u < 4; ++u) yv[u] = s_lut[(w >> (8 * u)) & 255u];
            } else {
                const float4 y4 = *reinterpret_cast<const float4 *>(y_all + o);
                yv[0] = y4.x; yv[1] = y4.y; yv[2] = y4.z; yv[3] = y4.w;
            }
            float g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                l1 += fabsf(xv[u] - yv[u]);
                g[u] = xv[u] > yv[u] ? l1_scale : (xv[u] < yv[u] ? -l1_scale : 0.f);
            }
            *reinterpret_cast<float4 *>(dL_drgb + o) = make_float4(g[0], g[1], g[2], g[3]);
            if (m_all) {
                const float4 m4 = *reinterpret_cast<const float4 *>(m_all + o);
                const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
                float gm[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    gm[u] = 0.f;
                    if (hit[u]) {
                        const float d = yv[u] - mv[u];
                        lt = fmaf(mt[u] * d, d, lt);
                        gm[u] = mesh_grad_scale * mt[u] * -d;
                    }
                }
                *reinterpret_cast<float4 *>(dL_dmesh + o) = make_float4(gm[0], gm[1], gm[2], gm[3]);
            }
        }
    }
    double sums[3] = {(double)l1, 0.0, (double)lt};
    block_sum3(sums, s_red);
    if (threadIdx.x < 3) partials[3 * (long long)blockIdx.x + threadIdx.x] = s_red[threadIdx.x][0];
}

// first level of the SSIM path's reduction (one partial per tile and channel,
// tens of thousands): CTA b sums partials [b kChunk, (b + 1) kChunk) into
// out[3 b .. 3 b + 2], so the FP64 additions spread over many SMs; the
// partition is fixed, so the order is the same on every call
constexpr int kChunk = 512;
__global__ void __launch_bounds__(kNT)
loss_reduce_kernel(const double *__restrict__ partials, int n_part, double *__restrict__ out) {
    __shared__ double s_red[3][kNT / 32];
    double v[3] = {0.0, 0.0, 0.0};
    const int lo = blockIdx.x * kChunk, hi = min(n_part, lo + kChunk);
    for (int i = lo + threadIdx.x; i < hi; i += kNT)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] += partials[3 * (long long)i + q];
    block_sum3(v, s_red);
    if (threadIdx.x < 3) out[3 * blockIdx.x + threadIdx.x] = s_red[threadIdx.x][0];
}

// one CTA: each thread sums a strided subset of the CTA partials, then a
// fixed-shape tree -- the same order on every call
__global__ void __launch_bounds__(kNT)
loss_final_kernel(const double *__restrict__ partials, int n_part, double inv_n, double ls, double lt,
                  double *__restrict__ out) {
    __shared__ double s_red[3][kNT / 32];
    double v[3] = {0.0, 0.0, 0.0};
    // eight strided partials loaded before they are added (in the same order
    // as one at a time): the loads overlap instead of serialising
    constexpr int kDepth = 8;
    int i = threadIdx.x;
    for (; i + (kDepth - 1) * kNT < n_part; i += kDepth * kNT) {
        double b[kDepth][3];
#pragma unroll
        for (int d = 0; d < kDepth; ++d)
#pragma unroll
            for (int q = 0; q < 3; ++q) b[d][q] = partials[3 * (long long)(i + d * kNT) + q];
#pragma unroll
        for (int d = 0; d < kDepth; ++d)
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] += b[d][q];
    }
    for (; i < n_part; i += kNT)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] += partials[3 * (long long)i + q];
    block_sum3(v, s_red);
    if (threadIdx.x == 0) {
        const double l1 = v[0] * inv_n, ss = v[1] * inv_n, t = v[2] * inv_n;
        out[0] = l1;
        out[1] = ss;
        out[2] = t;
        out[3] = (1.0 - ls) * l1 + ls * (1.0 - ss) + lt * t;
    }
}

// 8-bit image codes to [0, 1]: 16 codes per thread step (one uint4 load,
// four float4 stores), the ragged tail one by one
__global__ void __launch_bounds__(kNT)
decode_u8_kernel(const uint8_t *__restrict__ src, long long n, float *__restrict__ dst) {
    const long long n16 = n / 16;
    const uint4 *s16 = reinterpret_cast<const uint4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (long long i = (long long)blockIdx.x * kNT + threadIdx.x; i < n16; i += (long long)gridDim.x * kNT) {
        const uint4 w = s16[i];
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float f[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) f[b] = __fdiv_rn((float)((ww[q] >> (8 * b)) & 0xFFu), 255.f);
            d4[4 * i + q] = make_float4(f[0], f[1], f[2], f[3]);
        }
    }
    for (long long i = 16 * n16 + (long long)blockIdx.x * kNT + threadIdx.x; i < n; i += (long long)gridDim.x * kNT)
        dst[i] = __fdiv_rn((float)src[i], 255.f);
}

// the camera table with kLT x kLT loss tiles (validated as 16 x 16 render
// tiles, then re-tiled)
bool loss_view_table(const hm_camera *cams, int32_t n_views, ViewTable *vt) {
    hm_options o;
    hm_default_options(&o);
    o.tile_w = o.tile_h = 16;
    if (!build_view_table(cams, n_views, &o, vt)) return false;
    vt->tile_w = vt->tile_h = kLT;
    int tiles = 0;
    for (int v = 0; v < vt->n_views; ++v) {
        ViewDev &d = vt->v[v];
        d.tiles_x = (d.W + kLT - 1) / kLT;
        d.tiles_y = (d.H + kLT - 1) / kLT;
        d.tile_off = tiles;
        tiles += d.tiles_x * d.tiles_y;
    }
    vt->total_tiles = tiles;
    return true;
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
    return sizeof(float) * 9 * (size_t)vt.total_pixels + sizeof(double) * 9 * (size_t)vt.total_tiles + 4 * 256;
}

namespace hm {
namespace {

// the joint loss with FP32 targets or 8-bit target codes (TT = float or uint8_t)
template <typename TT>
hm_status hybrid_loss(const hm_camera *cams, int32_t n_views, const float *out_rgb, const TT *target,
                      const float *mesh_rgb, const float *out_T, const float *mesh_depth,
                      const hm_loss_params *p, double *loss_out, float *dL_drgb, float *dL_dmesh, void *ws,
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
    float2 *d_mu_xx = c.take<float2>(np3);
    float *d_xy = c.take<float>(np3);
    double *partials = c.take<double>(9 * (size_t)vt.total_tiles);
    cudaError_t e;
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
    if (p->lambda_ssim == 0.f) {
        // no SSIM term: one pointwise pass; mean SSIM is reported as 0
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long blocks = (vt.total_pixels + kNT - 1) / kNT;
        long long g1l = blocks < 8LL * sms ? blocks : 8LL * sms;
        if (g1l > 3LL * vt.total_tiles) g1l = 3LL * vt.total_tiles;   // the partials buffer holds 3 per tile
        const int g1 = (int)g1l;
        // four pixels a thread where every plane starts on a 16-byte boundary
        bool quad = (((uintptr_t)out_rgb | (uintptr_t)dL_drgb) & 15) == 0 &&
                    ((uintptr_t)target & (sizeof(TT) == 1 ? 3 : 15)) == 0;
        if (mesh)
            quad = quad && (((uintptr_t)mesh_rgb | (uintptr_t)out_T | (uintptr_t)mesh_depth | (uintptr_t)dL_dmesh) & 15) == 0;
        for (int v = 0; v < vt.n_views; ++v) quad = quad && ((long long)vt.v[v].W * vt.v[v].H) % 4 == 0;
        if (quad)
            l1_loss4_kernel<<<g1, kNT, 0, s>>>(vt, out_rgb, target, mesh ? mesh_rgb : nullptr, out_T, mesh_depth, p->k,
                                               (float)(1.0 / n_el), (float)(2.0 * p->lambda_t / n_el), dL_drgb,
                                               dL_dmesh, partials);
        else
            l1_loss_kernel<<<g1, kNT, 0, s>>>(vt, out_rgb, target, mesh ? mesh_rgb : nullptr, out_T, mesh_depth, p->k,
                                              (float)(1.0 / n_el), (float)(2.0 * p->lambda_t / n_el), dL_drgb,
                                              dL_dmesh, partials);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
        loss_final_kernel<<<1, kNT, 0, s>>>(partials, g1, 1.0 / n_el, 0.0, p->lambda_t, loss_out);
        return cuda_status(cudaGetLastError());
    }
    dim3 grid(vt.total_tiles, 3);
    ssim_fwd_kernel<<<grid, kNT, 0, s>>>(vt, tp, out_rgb, target, mesh ? mesh_rgb : nullptr, out_T,
                                               mesh_depth, p->k, (float)(2.0 * p->lambda_t / n_el), d_mu_xx,
                                         d_xy, dL_dmesh, partials);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    ssim_bwd_kernel<<<grid, kNT, 0, s>>>(vt, tp, out_rgb, target, d_mu_xx, d_xy,
                                               (float)((1.0 - p->lambda_ssim) / n_el),
                                               (float)(p->lambda_ssim / n_el), dL_drgb);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    const int n_part = 3 * vt.total_tiles, n_red = (n_part + kChunk - 1) / kChunk;
    double *level2 = partials + 3 * (size_t)n_part;     // 3 n_red <= 6 total_tiles doubles
    loss_reduce_kernel<<<n_red, kNT, 0, s>>>(partials, n_part, level2);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    loss_final_kernel<<<1, kNT, 0, s>>>(level2, n_red, 1.0 / n_el, p->lambda_ssim, p->lambda_t, loss_out);
    return cuda_status(cudaGetLastError());
}

}  // namespace
}  // namespace hm

extern "C" hm_status hm_hybrid_loss(const hm_camera *cams, int32_t n_views, const float *out_rgb,
                                    const float *target, const float *mesh_rgb, const float *out_T,
                                    const float *mesh_depth, const hm_loss_params *p,
                                    double *loss_out, float *dL_drgb, float *dL_dmesh, void *ws,
                                    size_t ws_bytes, void *stream) {
    return hybrid_loss(cams, n_views, out_rgb, target, mesh_rgb, out_T, mesh_depth, p, loss_out, dL_drgb,
                       dL_dmesh, ws, ws_bytes, stream);
}

extern "C" hm_status hm_hybrid_loss_u8(const hm_camera *cams, int32_t n_views, const float *out_rgb,
                                       const uint8_t *target, const float *mesh_rgb, const float *out_T,
                                       const float *mesh_depth, const hm_loss_params *p,
                                       double *loss_out, float *dL_drgb, float *dL_dmesh, void *ws,
                                       size_t ws_bytes, void *stream) {
    return hybrid_loss(cams, n_views, out_rgb, target, mesh_rgb, out_T, mesh_depth, p, loss_out, dL_drgb,
                       dL_dmesh, ws, ws_bytes, stream);
}

extern "C" hm_status hm_decode_u8(const uint8_t *src, int64_t n, float *dst, void *stream) {
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return HM_OK;
    if (!src || !dst) return fail(HM_ERR_INVALID_ARG, "null pointer");
    if (((uintptr_t)src & 15) || ((uintptr_t)dst & 15))
        return fail(HM_ERR_INVALID_ARG, "src and dst must be 16-byte aligned");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long need = (n / 16 + kNT - 1) / kNT + 1;
    const int grid = (int)(need < 8LL * sms ? need : 8LL * sms);
    decode_u8_kernel<<<grid, kNT, 0, (cudaStream_t)stream>>>(src, n, dst);
    return cuda_status(cudaGetLastError());
}
