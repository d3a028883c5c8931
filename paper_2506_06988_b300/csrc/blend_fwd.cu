// blend_fwd.cu -- hybrid front-to-back blending (Eq. 2 with the mesh cut-off
// and composite of Sec. 3.4).
//
// One CTA per screen tile, one thread per pixel.  The tile's depth-sorted
// list is consumed in batches: each batch's records are gathered once into
// shared memory and then evaluated by every pixel of the tile.  A pixel
// stops at the first Gaussian at or behind its mesh depth (the list is
// depth-ordered, so all later ones are behind too) or when T would fall below
// 1e-4; the CTA leaves the list as soon as every pixel has stopped
// (__syncthreads_count vote), which is where the opaque mesh shortens the
// per-pixel work.
//
// Per evaluated (pixel, Gaussian): q = -log2(e)/2 * d^2 from the pre-scaled
// conic (5 FP32 ops), one ex2, the alpha/T updates and three FMAs of colour.
#include "blend_common.cuh"
#include "hm_host.h"

namespace hm {

namespace {

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH)
blend_fwd_kernel(ViewTable vt, const Record *__restrict__ rec, const uint32_t *__restrict__ vals,
                 const uint32_t *__restrict__ ranges, const float *__restrict__ mesh_depth,
                 const float *__restrict__ mesh_rgb, float bg0, float bg1, float bg2, int batch,
                 float *__restrict__ out_rgb, float *__restrict__ out_T,
                 uint32_t *__restrict__ n_contrib, uint32_t *__restrict__ last_idx,
                 unsigned long long *__restrict__ eval_stats) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_a[NT];   // mean x, mean y, K*conic_xx, 2K*conic_xy
    __shared__ float4 s_b[NT];   // K*conic_yy, opacity, depth, -
    __shared__ float4 s_c[NT];   // r, g, b, -
    const int gt = blockIdx.x;
    const int v = view_of_tile(vt, gt);
    const ViewDev &V = vt.v[v];
    const int local = gt - V.tile_off;
    const int tx = local % V.tiles_x, ty = local / V.tiles_x;
    const int t = threadIdx.x;
    const int px = tx * TW + (t % TW), py = ty * TH + (t / TW);
    const bool inside = px < V.W && py < V.H;
    const long long npx = (long long)V.W * V.H;
    const long long lp = (long long)py * V.W + px;
    const long long gp = V.pix_off + lp;
    float Dm = INFINITY;
    float back0 = bg0, back1 = bg1, back2 = bg2;
    if (inside) {
        if (mesh_depth) Dm = mesh_depth[gp];
        if (mesh_rgb) {
            const float *m = mesh_rgb + 3 * V.pix_off + lp;
            back0 = m[0];
            back1 = m[npx];
            back2 = m[2 * npx];
        }
    }
    const uint32_t begin = ranges[2 * gt], end = ranges[2 * gt + 1];
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    bool done = !inside;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t cnt = 0, last = 0, n_eval = 0, n_exam = 0;
    for (uint32_t b0 = begin; b0 < end; b0 += batch) {
        if (__syncthreads_count(done) == NT) break;
        const uint32_t j = b0 + t;
        if (t < batch && j < end) {
            stage_record(rec[vals[j]], s_a[t], s_b[t], s_c[t]);
        }
        __syncthreads();
        if (!done) {
            const int nb = (int)min((uint32_t)batch, end - b0);
            for (int k = 0; k < nb; ++k) {
                const float4 A = s_a[k];
                const float4 B = s_b[k];
                if (B.z >= Dm) { done = true; break; }        // at or behind the mesh
                float dx, dy;
                const float q = eval_q(A, B, fpx, fpy, dx, dy);
                if (eval_stats) ++n_exam;
                if (q < kQ3) continue;                          // outside the 3-sigma ellipse
                if (eval_stats) ++n_eval;
                const float alpha = fminf(kAlphaMax, __fmul_rn(B.y, ex2_approx(q)));
                if (alpha < kAlphaMin) continue;
                const float Tn = T * (1.f - alpha);
                if (Tn < kTMin) { done = true; break; }
                const float w = alpha * T;
                const float4 c = s_c[k];
                C0 = fmaf(w, c.x, C0);
                C1 = fmaf(w, c.y, C1);
                C2 = fmaf(w, c.z, C2);
                T = Tn;
                ++cnt;
                last = b0 + k + 1;
            }
        }
    }
    if (inside) {
        float *o = out_rgb + 3 * V.pix_off + lp;
        o[0] = fmaf(T, back0, C0);
        o[npx] = fmaf(T, back1, C1);
        o[2 * npx] = fmaf(T, back2, C2);
        out_T[gp] = T;
        n_contrib[gp] = cnt;
        if (last_idx) last_idx[gp] = last;
    }
    if (eval_stats) {
        unsigned long long e = n_eval, x = n_exam;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            x += __shfl_xor_sync(0xffffffffu, x, o);
        }
        if ((t & 31) == 0) {
            atomicAdd(eval_stats, e);
            atomicAdd(eval_stats + 1, x);
        }
    }
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" hm_status hm_blend_forward(const hm_camera *cams, int32_t n_views, int32_t n,
                                      const void *records, const uint32_t *pair_vals,
                                      const uint32_t *tile_ranges, const float *mesh_depth,
                                      const float *mesh_rgb, const hm_options *opt,
                                      float *out_rgb, float *out_T, uint32_t *n_contrib,
                                      uint32_t *last_idx, unsigned long long *eval_stats,
                                      void *stream) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt)) return HM_ERR_INVALID_ARG;
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    const int nt = opt->tile_w * opt->tile_h;
    if (opt->batch < 1 || opt->batch > nt)
        return fail(HM_ERR_INVALID_ARG, "batch must be in 1..%d for this tile shape", nt);
    if (!tile_ranges || !out_rgb || !out_T || !n_contrib || (n > 0 && (!records || !pair_vals)))
        return fail(HM_ERR_INVALID_ARG, "null pointer");
    if ((uintptr_t)records & 15) return fail(HM_ERR_INVALID_ARG, "records must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const Record *rec = reinterpret_cast<const Record *>(records);
    dim3 grid(vt.total_tiles);
    const float *bg = opt->bg;
#define HM_BLEND(TW, TH)                                                                        \
    blend_fwd_kernel<TW, TH><<<grid, TW * TH, 0, s>>>(vt, rec, pair_vals, tile_ranges, mesh_depth, \
                                                      mesh_rgb, bg[0], bg[1], bg[2], opt->batch,   \
                                                      out_rgb, out_T, n_contrib, last_idx, eval_stats)
    if (opt->tile_w == 16) HM_BLEND(16, 16);
    else if (opt->tile_w == 32) HM_BLEND(32, 8);
    else HM_BLEND(8, 8);
#undef HM_BLEND
    return cuda_status(cudaGetLastError());
}
