// blend_fwd.cu -- hybrid front-to-back blending (Eq. 2 with the mesh cut-off
// and composite of Sec. 3.4).
//
// One CTA per screen tile; a thread owns two pixels of one column (rows y and
// y + 4 of its warp's 8x8 block), so the staged record, dx and the loop are
// shared by the pair and the pair's arithmetic runs in packed FP32x2
// (Blackwell FFMA2/FMUL2).  The tile's depth-sorted list is consumed in
// rounds of `batch` entries.  Each round's 48-byte records are fetched into
// shared memory by bulk asynchronous copies (cp.async.bulk, the TMA unit),
// one per entry, completing on the round's mbarrier; rounds are double
// buffered, so round r+1 is in flight while round r is evaluated, and the
// record indices of round r+2 are loaded meanwhile.  A pixel stops at the
// first Gaussian at or behind its mesh depth (the list is depth-ordered, so
// all later ones are behind too) or when T would fall below 1e-4; the CTA
// leaves the list as soon as every pixel has stopped (__syncthreads_count
// vote), which is where the opaque mesh shortens the per-pixel work.
//
// Per evaluated (pixel, Gaussian): q = -log2(e)/2 * d^2 from the record's
// pre-scaled conic, one ex2, the alpha/T updates and three FMAs of colour;
// updates are masked (alpha 0 for a pixel that does not blend) instead of
// branched, for entries outside the 3-sigma ellipse too.  A pixel's only
// loop-carried stop state is its cut depth: the mesh depth, or -inf once it
// lies outside the image or its T would fall below 1e-4.
#include "blend_common.cuh"
#include "hm_host.h"
#include "tma.cuh"

namespace hm {

namespace {

// Grid launch (PERSIST false): one CTA per tile.  Persistent launch: a grid
// of resident CTAs that claim tiles of all views from the counter `work`
// (zeroed before the launch) until none is left -- the (view, tile) work
// queue.  A claim is one atomic on a counter that only grows, so no CTA
// waits on another.
template <int TW, int TH, bool COUNT, bool PERSIST>
__global__ void __launch_bounds__(TW *TH / 2, 8)
blend_fwd_kernel(ViewTable vt, const Record *__restrict__ rec, uint32_t n_rec,
                 const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
                 const float *__restrict__ mesh_depth, const float *__restrict__ mesh_rgb, float bg0,
                 float bg1, float bg2, int batch, float *__restrict__ out_rgb,
                 float *__restrict__ out_T, uint32_t *__restrict__ n_contrib,
                 uint32_t *__restrict__ last_idx, unsigned long long *__restrict__ eval_stats,
                 int32_t *__restrict__ d_status, unsigned int *__restrict__ work) {
    __shared__ Record s_rec[2][TW * TH];
    __shared__ uint64_t s_bar[2];
    __shared__ int s_tile, s_timeout;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
    }
    uint32_t ph0 = 0u, ph1 = 0u;
    // One tile: the whole Eq. 2 walk of its pixels.  ph0 / ph1 count the phases
    // of barrier 0 / 1 completed before this tile (the wait parity of round r is
    // (ph_{r & 1} + r / 2) & 1); every round issued here is waited for before the
    // return, so the counts stay exact.  With PERSIST, returns false
    // (block-uniform) after a timed-out wait: the barriers' phases are then
    // unknown and the CTA claims no more tiles.
    auto blend_tile = [&](const int gt) -> bool {
        constexpr int NT = TW * TH, NTH = NT / 2;
        const int v = view_of_tile(vt, gt);
        const ViewDev &V = vt.v[v];
        const int local = gt - V.tile_off;
        const int tx = local % V.tiles_x, ty = local / V.tiles_x;
        const int t = threadIdx.x;
        int px, pya, pyb;
        pixel_pair<TW>(t, tx * TW, ty * TH, px, pya, pyb);
        const bool in_a = px < V.W && pya < V.H, in_b = px < V.W && pyb < V.H;
        const long long npx = (long long)V.W * V.H;
        const long long lpa = (long long)pya * V.W + px, lpb = (long long)pyb * V.W + px;
        uint32_t begin = ranges[2 * gt], end = ranges[2 * gt + 1];
        if (!hm_check(begin <= end)) begin = end = 0;   // (checked build: an inverted range is empty)
        const uint32_t n_rounds = end > begin ? (end - begin + (uint32_t)batch - 1) / (uint32_t)batch : 0u;
        // wait parity of round r (the grid launch starts every barrier at phase 0)
        auto parity = [&](uint32_t r) -> uint32_t {
            if constexpr (PERSIST) return (((r & 1) ? ph1 : ph0) + (r >> 1)) & 1u;
            else return (r >> 1) & 1u;
        };
        if constexpr (PERSIST)
            if (t == 0) s_timeout = 0;                    // published by the barrier before the first issue
        // record indices of the next round to issue (entries t and t + NTH)
        uint32_t nxt0 = 0, nxt1 = 0;
        auto load_idx = [&](uint32_t r) {
            const uint32_t b0 = begin + r * (uint32_t)batch;
            const uint32_t nb = min((uint32_t)batch, end - b0);
            if ((uint32_t)t < nb) nxt0 = vals[b0 + t];
            if ((uint32_t)(t + NTH) < nb) nxt1 = vals[b0 + t + NTH];
        };
        auto issue = [&](uint32_t r) {
            const int buf = r & 1;
            const uint32_t b0 = begin + r * (uint32_t)batch;
            const uint32_t nb = min((uint32_t)batch, end - b0);
            if (t == 0) mbar_arrive_expect_tx(&s_bar[buf], nb * (uint32_t)sizeof(Record));
            if ((uint32_t)t < nb) {
                uint32_t it = nxt0;
                if (it >= n_rec) { set_status(d_status, HM_DEV_BAD_INDEX); it = 0; }
                bulk_g2s(&s_rec[buf][t], rec + it, sizeof(Record), &s_bar[buf]);
            }
            if ((uint32_t)(t + NTH) < nb) {
                uint32_t it = nxt1;
                if (it >= n_rec) { set_status(d_status, HM_DEV_BAD_INDEX); it = 0; }
                bulk_g2s(&s_rec[buf][t + NTH], rec + it, sizeof(Record), &s_bar[buf]);
            }
        };
        if (n_rounds > 0) load_idx(0);
        __syncthreads();                                 // barriers initialised
        if (n_rounds > 0) issue(0);
        if (n_rounds > 1) load_idx(1);

        float Dm_a = INFINITY, Dm_b = INFINITY;
        if (mesh_depth) {
            if (in_a) Dm_a = mesh_depth[V.pix_off + lpa];
            if (in_b) Dm_b = mesh_depth[V.pix_off + lpb];
        }
        const float fpx = (float)px + 0.5f;
        const float2 fpy = make_float2((float)pya + 0.5f, (float)pyb + 0.5f);
        // a pixel takes entries with depth < Dm (the list is depth-ordered, so
        // the first entry at or behind the mesh ends it); outside the image,
        // or once its T would fall below 1e-4, Dm is -inf
        if (!in_a) Dm_a = -INFINITY;
        if (!in_b) Dm_b = -INFINITY;
        bool stopped = false;                            // this thread has left the list
        float2 T = make_float2(1.f, 1.f);
        float2 C0 = make_float2(0.f, 0.f), C1 = C0, C2 = C0;
        uint32_t cnt_a = 0, cnt_b = 0, last_a = 0, last_b = 0, n_eval = 0, n_exam = 0;
        uint32_t issued = n_rounds > 0 ? 1u : 0u, consumed = 0;
        bool all_landed = true;                          // persistent launch only
        for (uint32_t r = 0; r < n_rounds; ++r) {
            // every pixel has stopped (or, in the persistent launch, a wait of the
            // CTA timed out): leave the list.  The barrier also ends every
            // thread's reads of round r - 1, whose buffer round r + 1 refills.
            if constexpr (PERSIST) {
                if (__syncthreads_count(stopped) == NTH || s_timeout) break;
            } else {
                if (__syncthreads_count(stopped) == NTH) break;
            }
            if (r + 1 < n_rounds) {
                issue(r + 1);
                ++issued;
                if (r + 2 < n_rounds) load_idx(r + 2);
            }
            const int buf = r & 1;
            if (!mbar_wait(&s_bar[buf], parity(r))) {
                set_status(d_status, HM_DEV_TIMEOUT);
                if constexpr (PERSIST) {
                    all_landed = false;
                    s_timeout = 1;
                }
                stopped = true;
            }
            consumed = r + 1;
            if (stopped) continue;
            const uint32_t b0 = begin + r * (uint32_t)batch;
            const int nb = (int)min((uint32_t)batch, end - b0);
            const Record *sr = s_rec[buf];
            for (int k = 0; k < nb; ++k) {
                const float4 B = sr[k].b;
                // at or behind the mesh: this and every later Gaussian is cut
                const bool la = B.z < Dm_a, lb = B.z < Dm_b;
                if (!(la || lb)) {
                    stopped = true;
                    break;
                }
                const float4 A = sr[k].a;
                float dx;
                float2 dy;
                const float2 q = eval_q2(A, B, fpx, fpy, dx, dy);
                bool ea = la && q.x >= kQ3, eb = lb && q.y >= kQ3;   // inside the 3-sigma ellipse
                if (COUNT) n_exam += la + lb, n_eval += ea + eb;
                float2 G, araw;
                const float2 al = eval_alpha2(B.y, q, G, araw);
                ea = ea && al.x >= kAlphaMin;
                eb = eb && al.y >= kAlphaMin;
                const float2 Tn = __ffma2_rn(make_float2(-T.x, -T.y), al, T);   // T (1 - alpha)
                // stop before a Gaussian that would take T below 1e-4
                if (ea && Tn.x < kTMin) { Dm_a = -INFINITY; ea = false; }
                if (eb && Tn.y < kTMin) { Dm_b = -INFINITY; eb = false; }
                const float2 ae = make_float2(ea ? al.x : 0.f, eb ? al.y : 0.f);
                const float2 w = __fmul2_rn(ae, T);
                const float4 c = sr[k].c;
                C0 = __ffma2_rn(w, make_float2(c.x, c.x), C0);
                C1 = __ffma2_rn(w, make_float2(c.y, c.y), C1);
                C2 = __ffma2_rn(w, make_float2(c.z, c.z), C2);
                T = __ffma2_rn(make_float2(-T.x, -T.y), ae, T);     // Tn where blended, T where ae = 0
                cnt_a += ea;
                cnt_b += eb;
                if (ea) last_a = b0 + k + 1;
                if (eb) last_b = b0 + k + 1;
            }
        }
        // a round issued but not consumed (early exit), and the last one
        // waited for (its wait may have timed out), must land before the
        // buffers are reused or the CTA's shared memory is released; waiting
        // again for a round that has landed returns at once (its barrier's
        // next phase on the same buffer is not issued before it is consumed)
        bool drained = true;
        if (t == 0) {
            for (uint32_t r = consumed > 0 ? consumed - 1 : 0; r < issued; ++r)
                if (!mbar_wait(&s_bar[r & 1], parity(r))) {
                    set_status(d_status, HM_DEV_TIMEOUT);
                    drained = false;
                }
        }
        if constexpr (PERSIST) {
            ph0 += (issued + 1) >> 1;                    // rounds 0, 2, 4, ... used barrier 0
            ph1 += issued >> 1;
        }
        const float *mr = mesh_rgb ? mesh_rgb + 3 * V.pix_off : nullptr;
        float *o = out_rgb + 3 * V.pix_off;
        if (in_a) {
            o[lpa] = fmaf(T.x, mr ? mr[lpa] : bg0, C0.x);
            o[npx + lpa] = fmaf(T.x, mr ? mr[npx + lpa] : bg1, C1.x);
            o[2 * npx + lpa] = fmaf(T.x, mr ? mr[2 * npx + lpa] : bg2, C2.x);
            out_T[V.pix_off + lpa] = T.x;
            n_contrib[V.pix_off + lpa] = cnt_a;
            if (last_idx) last_idx[V.pix_off + lpa] = last_a;
        }
        if (in_b) {
            o[lpb] = fmaf(T.y, mr ? mr[lpb] : bg0, C0.y);
            o[npx + lpb] = fmaf(T.y, mr ? mr[npx + lpb] : bg1, C1.y);
            o[2 * npx + lpb] = fmaf(T.y, mr ? mr[2 * npx + lpb] : bg2, C2.y);
            out_T[V.pix_off + lpb] = T.y;
            n_contrib[V.pix_off + lpb] = cnt_b;
            if (last_idx) last_idx[V.pix_off + lpb] = last_b;
        }
        if (COUNT) {
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
        if constexpr (PERSIST) return __syncthreads_and(all_landed && drained);
        return true;
    };
    if constexpr (!PERSIST) {
        // (the tile's first barrier publishes the barrier initialisation)
        blend_tile(blockIdx.x);
    } else {
        for (;;) {
            __syncthreads();                              // the previous tile's shared reads are done
            if (threadIdx.x == 0) s_tile = (int)atomicAdd(work, 1u);
            __syncthreads();
            const int gt = s_tile;
            if (gt >= vt.total_tiles) return;
            if (!blend_tile(gt)) return;                  // a wait timed out: phases unknown, stop claiming
        }
    }
}

}  // namespace

// resident CTAs per SM of a kernel at a block size (cached per device)
template <typename K>
int resident_ctas(K kernel, int threads, int slot) {
    static int cache[64][8] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int &c = cache[dev][slot];
    if (c == 0) {
        int per_sm = 0, nsm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        c = per_sm * nsm;
    }
    return c;
}

}  // namespace hm

using namespace hm;

extern "C" hm_status hm_blend_forward(const hm_camera *cams, int32_t n_views, int32_t n,
                                      const void *records, const uint32_t *pair_vals,
                                      const uint32_t *tile_ranges, const float *mesh_depth,
                                      const float *mesh_rgb, const hm_options *opt,
                                      float *out_rgb, float *out_T, uint32_t *n_contrib,
                                      uint32_t *last_idx, unsigned long long *eval_stats,
                                      int32_t *d_status, uint32_t *work, void *stream) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt)) return HM_ERR_INVALID_ARG;
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    const int nt = opt->tile_w * opt->tile_h;
    if (opt->batch < 1 || opt->batch > nt)
        return fail(HM_ERR_INVALID_ARG, "batch must be in 1..%d for this tile shape", nt);
    if (!tile_ranges || !out_rgb || !out_T || !n_contrib || (n > 0 && (!records || !pair_vals)))
        return fail(HM_ERR_INVALID_ARG, "null pointer");
    if ((uintptr_t)records & 15) return fail(HM_ERR_INVALID_ARG, "records must be 16-byte aligned");
    if (opt->persistent && (!work || ((uintptr_t)work & 3)))
        return fail(HM_ERR_INVALID_ARG, "a persistent launch needs a 4-byte aligned work counter");
    cudaStream_t s = (cudaStream_t)stream;
    const Record *rec = reinterpret_cast<const Record *>(records);
    const float *bg = opt->bg;
    unsigned int *wq = opt->persistent ? reinterpret_cast<unsigned int *>(work) : nullptr;
    if (wq) {
        const cudaError_t e = cudaMemsetAsync(wq, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return cuda_status(e);
    }
#define HM_BLEND(TW, TH, SLOT)                                                                        \
    do {                                                                                              \
        auto kern = wq ? (eval_stats ? blend_fwd_kernel<TW, TH, true, true>                           \
                                     : blend_fwd_kernel<TW, TH, false, true>)                         \
                       : (eval_stats ? blend_fwd_kernel<TW, TH, true, false>                          \
                                     : blend_fwd_kernel<TW, TH, false, false>);                       \
        int grid = vt.total_tiles;                                                                    \
        if (wq) {                                                                                     \
            grid = resident_ctas(kern, TW * TH / 2, SLOT + (eval_stats ? 1 : 0));                     \
            if (grid <= 0) return fail(HM_ERR_CUDA, "occupancy query failed");                        \
            grid = grid < vt.total_tiles ? grid : vt.total_tiles;                                     \
        }                                                                                             \
        kern<<<grid, TW * TH / 2, 0, s>>>(vt, rec, n_rec, pair_vals, tile_ranges, mesh_depth,         \
                                          mesh_rgb, bg[0], bg[1], bg[2], opt->batch, out_rgb, out_T,  \
                                          n_contrib, last_idx, eval_stats, d_status, wq);             \
    } while (0)
    const uint32_t n_rec = (uint32_t)((long long)n_views * n);
    if (vt.total_tiles > 0) {
        if (opt->tile_w == 16) HM_BLEND(16, 16, 0);
        else if (opt->tile_w == 32) HM_BLEND(32, 8, 2);
        else HM_BLEND(8, 8, 4);
    }
#undef HM_BLEND
    return cuda_status(cudaGetLastError());
}

#ifdef HM_CHECKED
namespace hm {
HM_CHECKED_READER(blend_fwd)
}  // namespace hm
#endif
