// blend_bwd.cu -- gradients of the hybrid render (Eq. 2 blending with the
// Sec. 3.4 composite I_h = I_gs + T * back) with respect to the Gaussian
// parameters and the texels (the texture map is optimisable, Sec. 3.4).
//
// Three kernels:
//  * blend_bwd: per tile, per pixel (pixel pairs of a column in packed
//    FP32x2, as in the forward; two pairs per thread on 16x16 tiles), the
//    blended Gaussians are replayed back to front from the pixel's last
//    blended list position.  With
//    B = (colour behind Gaussian i) / T_{i+1}, running from B = back:
//        dI/dc_i     = alpha_i T_i
//        dI/dalpha_i = T_i (c_i - B),  dT_final/dalpha_i = -T_final/(1-alpha_i)
//        B <- alpha_i c_i + (1 - alpha_i) B,  T_i = T_{i+1} / (1 - alpha_i).
//    Decisions are re-evaluated with the forward's exact arithmetic
//    (blend_common.cuh).  Per Gaussian the 9 partials (five pixel-space
//    moments of dL/dq from which the mean2d and conic gradients follow,
//    opacity, colour) are summed over the thread's pixels and written to a
//    per-warp ring in shared memory; every three entries the warp sums each
//    (entry, value) column over its 32 lanes (one lane per column, packed
//    FP32x2 adds) and adds it to the record's accumulator with one atomic.
//  * texture_bwd: dL/dtexel += T * w_bilinear * dL/dI_h on pixels with a
//    triangle (the mesh colour enters I_h weighted by T), summed per screen
//    tile in shared memory (fixed point) before the global reductions.
//  * project_bwd: one thread per (Gaussian, view) pair with a gradient
//    turns the view's moments into dL/dmean2d and dL/dconic with the view's
//    conic and chains them through the conic inverse, Sigma' = V V^T,
//    V = (J W)(R S), the clamped Jacobian, the projection of the mean, the
//    quaternion normalisation and the SH colour (including its dependence
//    on the mean through the view direction); the views of a Gaussian add
//    their (linear) contributions with atomics.
#include <mutex>

#include "blend_common.cuh"
#include "hm_host.h"
#include "sh.cuh"
#include "tma.cuh"

namespace hm {

namespace {

// per-record partials left by the blend replay: the moments of dL/dq over the
// record's pixels (sum gq dx, sum gq dy, sum gq dx^2, sum gq dx dy,
// sum gq dy^2; q = K d^2, (dx, dy) = pixel centre - mean), dL/dopacity and
// dL/dcolour (r, g, b)
constexpr int kG = 9;
// list entries whose per-lane partials a warp of the replay collects before
// it sums them over its lanes (3 x 9 columns: one flush pass of 27 lanes)
constexpr int kRingEntries = 3;
// the replay's staging batch: at most this many list entries per round, so
// that the double-buffered records and the partials ring leave room for 12
// CTAs per SM
constexpr int kBwdBatchMax = 64;

// Pixel layout of the replay: a warp covers 8 columns x 8 PP rows of the
// tile; lane l owns column l % 8 and, for p < PP, the pixel pair of rows
// l / 8 + 8 p and l / 8 + 8 p + 4 (PP = 1 is the forward's layout).  With
// PP = 2 a thread holds two pairs of one column: the column part of q and
// the warp reduction of the nine partials are shared by four pixels.  The
// staged records live in dynamic shared memory sized by the batch.
// Grid launch (PERSIST false): one CTA per tile.  Persistent launch: a grid
// of resident CTAs that claim tiles of all views from the counter `work`
// (zeroed before the launch) until none is left; a claim is one atomic on a
// counter that only grows, so no CTA waits on another.
template <int TW, int TH, int PP, bool PERSIST, bool HAS_DT>
__global__ void __launch_bounds__(TW *TH / (2 * PP), PP == 1 ? 6 : 12)
blend_bwd_kernel(ViewTable vt, const Record *__restrict__ rec, uint32_t n_rec,
                 const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
                 const float *__restrict__ mesh_rgb, float bg0, float bg1, float bg2,
                 const float *__restrict__ out_T, const uint32_t *__restrict__ last_idx,
                 const float *__restrict__ dL_drgb, const float *__restrict__ dL_dT, int batch,
                 float *__restrict__ g2d, int32_t *__restrict__ d_status, unsigned int *__restrict__ work) {
    static_assert(TW % 8 == 0 && TH % (8 * PP) == 0, "tile shape");
    extern __shared__ __align__(16) unsigned char s_dyn[];
    Record *s_rec0 = reinterpret_cast<Record *>(s_dyn);              // [2][batch]
    uint32_t *s_item0 = reinterpret_cast<uint32_t *>(s_rec0 + 2 * batch);   // [2][batch]
    __shared__ uint64_t s_bar[2];
    __shared__ uint32_t s_hi;
    __shared__ int s_tile;
    // per-warp ring of the last RNE entries' per-lane partials: [entry][value][lane]
    // rows padded to RRS floats, so that the flush's 16-byte column reads by
    // eight lanes fall in distinct banks
    constexpr int RNE = kRingEntries, RRS = 36, NW = TW * TH / (2 * PP) / 32;
    static_assert(RNE * kG <= 32, "one flush pass");
    __shared__ __align__(16) float s_ring[NW][RNE][kG][RRS];
    __shared__ uint32_t s_ridx[NW][RNE];
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
    }
    uint32_t ph0 = 0u, ph1 = 0u;
    // One tile's replay.  ph0 / ph1 count the phases of barrier 0 / 1 completed
    // before this tile (the wait parity of round r is (ph_{r & 1} + r / 2) & 1);
    // every round issued here is waited for before the return.  Returns false
    // (block-uniform) after a timed-out wait.
    auto replay_tile = [&](const int gt) -> bool {
        constexpr int NTH = TW * TH / (2 * PP);
        constexpr int PER = (TW * TH + NTH - 1) / NTH;       // staged records per thread and round, at most
        const int v = view_of_tile(vt, gt);
        const ViewDev &V = vt.v[v];
        const int local = gt - V.tile_off;
        const int tx = local % V.tiles_x, ty = local / V.tiles_x;
        const int t = threadIdx.x, lane = t & 31;
        constexpr int WX = TW / 8;
        const int px = tx * TW + ((t >> 5) % WX) * 8 + (lane & 7);
        const int row0 = ty * TH + ((t >> 5) / WX) * (8 * PP) + (lane >> 3);
        const long long npx = (long long)V.W * V.H;
        const float *gI = dL_drgb + 3 * V.pix_off;
        const float *mr = mesh_rgb ? mesh_rgb + 3 * V.pix_off : nullptr;
        float2 Tf[PP], gI0[PP], gI1[PP], gI2[PP], gT[PP], B0[PP], B1[PP], B2[PP], fpy[PP];
        uint32_t la[PP], lb[PP];
        uint32_t my_hi = 0;
    #pragma unroll
        for (int p = 0; p < PP; ++p) {
            const int pya = row0 + 8 * p, pyb = pya + 4;
            const bool in_a = px < V.W && pya < V.H, in_b = px < V.W && pyb < V.H;
            const long long lpa = (long long)pya * V.W + px, lpb = (long long)pyb * V.W + px;
            Tf[p] = make_float2(1.f, 1.f);
            gI0[p] = gI1[p] = gI2[p] = gT[p] = make_float2(0.f, 0.f);
            B0[p] = make_float2(bg0, bg0);
            B1[p] = make_float2(bg1, bg1);
            B2[p] = make_float2(bg2, bg2);
            la[p] = lb[p] = 0;
            fpy[p] = make_float2((float)pya + 0.5f, (float)pyb + 0.5f);
            // a pixel that blended nothing has nothing to replay: its other
            // inputs are not read
            if (in_a) la[p] = last_idx[V.pix_off + lpa];
            if (in_b) lb[p] = last_idx[V.pix_off + lpb];
            if (la[p] > 0) {
                Tf[p].x = out_T[V.pix_off + lpa];
                gI0[p].x = gI[lpa]; gI1[p].x = gI[npx + lpa]; gI2[p].x = gI[2 * npx + lpa];
                if constexpr (HAS_DT) gT[p].x = dL_dT[V.pix_off + lpa];
                if (mr) { B0[p].x = mr[lpa]; B1[p].x = mr[npx + lpa]; B2[p].x = mr[2 * npx + lpa]; }
            }
            if (lb[p] > 0) {
                Tf[p].y = out_T[V.pix_off + lpb];
                gI0[p].y = gI[lpb]; gI1[p].y = gI[npx + lpb]; gI2[p].y = gI[2 * npx + lpb];
                if constexpr (HAS_DT) gT[p].y = dL_dT[V.pix_off + lpb];
                if (mr) { B0[p].y = mr[lpb]; B1[p].y = mr[npx + lpb]; B2[p].y = mr[2 * npx + lpb]; }
            }
            my_hi = max(my_hi, max(la[p], lb[p]));
        }
        const uint32_t begin = ranges[2 * gt];
        if (t == 0) s_hi = 0;
        __syncthreads();
        if (my_hi > 0) atomicMax(&s_hi, my_hi);
        __syncthreads();
        uint32_t hi_all = s_hi;
        // (checked build: stop positions must lie in the tile's list)
        if (!hm_check(hi_all == 0 || (begin <= hi_all && hi_all <= ranges[2 * gt + 1]))) hi_all = begin;
        // rounds walk the list back to front: round r covers [lo_r, hi_r) with
        // hi_r = hi_all - r batch, lo_r = max(begin, hi_r - batch)
        const uint32_t n_rounds = hi_all > begin ? (hi_all - begin + (uint32_t)batch - 1) / (uint32_t)batch : 0u;
        uint32_t nxt[PER];
    #pragma unroll
        for (int e = 0; e < PER; ++e) nxt[e] = 0;
        auto round_lo = [&](uint32_t r, uint32_t &lo, uint32_t &nb) {
            const uint32_t hi = hi_all - r * (uint32_t)batch;
            lo = hi - begin > (uint32_t)batch ? hi - (uint32_t)batch : begin;
            nb = hi - lo;
        };
        auto load_idx = [&](uint32_t r) {
            uint32_t lo, nb;
            round_lo(r, lo, nb);
    #pragma unroll
            for (int e = 0; e < PER; ++e)
                if ((uint32_t)(t + e * NTH) < nb) nxt[e] = vals[lo + t + e * NTH];
        };
        auto issue = [&](uint32_t r) {
            const int buf = r & 1;
            uint32_t lo, nb;
            round_lo(r, lo, nb);
            if (t == 0) mbar_arrive_expect_tx(&s_bar[buf], nb * (uint32_t)sizeof(Record));
    #pragma unroll
            for (int e = 0; e < PER; ++e) {
                const uint32_t k = (uint32_t)(t + e * NTH);
                if (k < nb) {
                    uint32_t it = nxt[e];
                    if (it >= n_rec) { set_status(d_status, HM_DEV_BAD_INDEX); it = 0; }
                    s_item0[buf * batch + k] = it;
                    bulk_g2s(&s_rec0[buf * batch + k], rec + it, sizeof(Record), &s_bar[buf]);
                }
            }
        };
        if (n_rounds > 0) {
            load_idx(0);
            issue(0);
        }
        if (n_rounds > 1) load_idx(1);
        // the ring's flush: lane c < n kG sums column (entry c / kG, value c % kG)
        // over the warp's 32 lanes and adds it to the record's partial
        const int wid = t >> 5;
        int nfill = 0;
        auto ring_flush = [&](int n) {
            __syncwarp();
            if (lane < n * kG) {
                const int e = lane / kG, v = lane - e * kG;
                const float4 *p = reinterpret_cast<const float4 *>(&s_ring[wid][e][v][0]);
                float2 acc[4];
    #pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 a = p[2 * j], b = p[2 * j + 1];
                    acc[j] = __fadd2_rn(__fadd2_rn(make_float2(a.x, a.y), make_float2(a.z, a.w)),
                                        __fadd2_rn(make_float2(b.x, b.y), make_float2(b.z, b.w)));
                }
                const float2 s2 = __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
                const float tot = s2.x + s2.y;
                if (tot != 0.f) atomicAdd(g2d + (size_t)s_ridx[wid][e] * kG + v, tot);
            }
            __syncwarp();
        };
        const float fpx = (float)px + 0.5f;
        float2 T[PP], gTT[PP];
    #pragma unroll
        for (int p = 0; p < PP; ++p) {
            T[p] = Tf[p];
            gTT[p] = __fmul2_rn(gT[p], Tf[p]);
        }
        bool ok = true;
        // rounds [consumed, issued) have copies that may still be in flight
        uint32_t issued = n_rounds > 0 ? 1u : 0u, consumed = 0;
        for (uint32_t r = 0; r < n_rounds; ++r) {
            // ends every thread's use of round r - 1, whose buffers round r + 1
            // refills, and publishes round r's record indices; after a timed-out
            // wait anywhere in the CTA nothing more is issued
            ok = __syncthreads_and(ok);
            if (!ok) break;
            if (r + 1 < n_rounds) {
                issue(r + 1);
                issued = r + 2;
                if (r + 2 < n_rounds) load_idx(r + 2);
            }
            const int buf = r & 1;
            if (!mbar_wait(&s_bar[buf], ((buf ? ph1 : ph0) + (r >> 1)) & 1u)) {
                set_status(d_status, HM_DEV_TIMEOUT);
                ok = false;
            }
            ok = __all_sync(0xffffffffu, ok);   // the replay below uses warp shuffles
            if (ok) consumed = r + 1;
            uint32_t lo, nb_u;
            round_lo(r, lo, nb_u);
            const int nb = ok ? (int)nb_u : 0;
            const Record *sr = s_rec0 + buf * batch;
            const uint32_t *si = s_item0 + buf * batch;
            for (int k = nb - 1; k >= 0; --k) {
                const uint32_t j = lo + k;
                bool ea[PP], eb[PP];
                bool act = false;
    #pragma unroll
                for (int p = 0; p < PP; ++p) {
                    ea[p] = j < la[p];
                    eb[p] = j < lb[p];
                    act = act || ea[p] || eb[p];
                }
                if (!__any_sync(0xffffffffu, act)) continue;
                const float4 A = sr[k].a, Bs = sr[k].b, c = sr[k].c;
                const QCol qc = eval_qcol(A, fpx);
                float2 dy[PP], ae[PP];
                bool actp[PP];
                act = false;
    #pragma unroll
                for (int p = 0; p < PP; ++p) {
                    const float2 q = eval_qrows(A, Bs, qc, fpy[p], dy[p]);
                    float2 G, araw;
                    const float2 al = eval_alpha2(Bs.y, q, G, araw);
                    // the forward blended it: alpha, else 0
                    const bool ba = ea[p] && q.x >= kQ3 && al.x >= kAlphaMin;
                    const bool bb = eb[p] && q.y >= kQ3 && al.y >= kAlphaMin;
                    ae[p] = make_float2(ba ? al.x : 0.f, bb ? al.y : 0.f);
                    // pair p of some lane blended it (warp-uniform)
                    actp[p] = __any_sync(0xffffffffu, ba || bb);
                    act = act || actp[p];
                }
                // entries the forward blended at none of the warp's pixels need no
                // gradient math and no reduction; within an entry, a pair row no
                // lane blended is skipped (its updates would be the identity)
                if (!act) continue;
                // per-record sums over the thread's pairs, packed (one horizontal
                // add per entry): dL/dq / ln 2 and its dy, dy^2 moments, dL/dcolour
                float2 s_gq = make_float2(0.f, 0.f), s_dy = s_gq, s_dy2 = s_gq, s_c0 = s_gq, s_c1 = s_gq,
                       s_c2 = s_gq;
    #pragma unroll
                for (int p = 0; p < PP; ++p) {
                    if (!actp[p]) continue;
                    // a pixel that did not blend the entry has alpha 0: 1 / (1 - 0) is
                    // exactly 1, so its T_i, B and sums pass through unchanged
                    const float2 om = __fadd2_rn(make_float2(1.f, 1.f), make_float2(-ae[p].x, -ae[p].y));
                    const float2 rr = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                    const float2 Ti = __fmul2_rn(T[p], rr);
                    // colour: dI/dc = alpha T_i
                    const float2 wgt = __fmul2_rn(ae[p], Ti);
                    s_c0 = __ffma2_rn(wgt, gI0[p], s_c0);
                    s_c1 = __ffma2_rn(wgt, gI1[p], s_c1);
                    s_c2 = __ffma2_rn(wgt, gI2[p], s_c2);
                    // dL/dalpha = T_i (gI . (c - B)) - dL/dT T_final / (1 - alpha)
                    const float2 d0 = __fadd2_rn(make_float2(c.x, c.x), make_float2(-B0[p].x, -B0[p].y));
                    const float2 d1 = __fadd2_rn(make_float2(c.y, c.y), make_float2(-B1[p].x, -B1[p].y));
                    const float2 d2 = __fadd2_rn(make_float2(c.z, c.z), make_float2(-B2[p].x, -B2[p].y));
                    float2 sdot = __fmul2_rn(gI0[p], d0);
                    sdot = __ffma2_rn(gI1[p], d1, sdot);
                    sdot = __ffma2_rn(gI2[p], d2, sdot);
                    float2 dLda = __fmul2_rn(Ti, sdot);
                    if constexpr (HAS_DT) dLda = __ffma2_rn(make_float2(-gTT[p].x, -gTT[p].y), rr, dLda);
                    // dL/dq / ln 2 = alpha dL/dalpha where blended and not clamped at
                    // 0.99 (a clamped alpha is exactly 0.99)
                    const float2 au = make_float2(ae[p].x < kAlphaMax ? ae[p].x : 0.f,
                                                  ae[p].y < kAlphaMax ? ae[p].y : 0.f);
                    // the pixel-space moments of dL/dq (the mean and conic
                    // gradients follow per record from them: dq/dmean = -2K conic
                    // (dx, dy), dq/dconic = K (dx^2, 2 dx dy, dy^2)); dx is shared
                    // by the thread's pixels.  The factor ln 2 is applied once per
                    // record in the projection backward
                    const float2 gq = __fmul2_rn(dLda, au);
                    const float2 gqdy = __fmul2_rn(gq, dy[p]);
                    s_gq = __fadd2_rn(s_gq, gq);
                    s_dy = __fadd2_rn(s_dy, gqdy);
                    s_dy2 = __ffma2_rn(gqdy, dy[p], s_dy2);
                    // colour behind the previous Gaussian (normalised):
                    // alpha c + (1 - alpha) B = B + alpha (c - B); then T_i
                    B0[p] = __ffma2_rn(ae[p], d0, B0[p]);
                    B1[p] = __ffma2_rn(ae[p], d1, B1[p]);
                    B2[p] = __ffma2_rn(ae[p], d2, B2[p]);
                    T[p] = Ti;
                }
                float g[kG];
                const float sgq = s_gq.x + s_gq.y;
                g[1] = s_dy.x + s_dy.y;
                g[4] = s_dy2.x + s_dy2.y;
                g[5] = sgq * rcp_approx(Bs.y);                               // dL/do = sum gq / o
                g[6] = s_c0.x + s_c0.y;
                g[7] = s_c1.x + s_c1.y;
                g[8] = s_c2.x + s_c2.y;
                g[0] = qc.dx * sgq;                                           // sum gq dx
                g[2] = qc.dx * g[0];                                          // sum gq dx^2
                g[3] = qc.dx * g[1];                                          // sum gq dx dy
                float *row = &s_ring[wid][nfill][0][0];
    #pragma unroll
                for (int v = 0; v < kG; ++v) row[v * RRS + lane] = g[v];
                if (lane == 0) s_ridx[wid][nfill] = si[k];
                if (++nfill == RNE) {
                    ring_flush(RNE);
                    nfill = 0;
                }
            }
        }
        if (nfill > 0) ring_flush(nfill);
        // after a timed-out wait, every copy issued and not yet waited for must
        // land (bounded waits) before the buffers are reused or the CTA's shared
        // memory is released
        ok = __syncthreads_and(ok);
        if (!ok && t == 0) {
            for (uint32_t r = consumed; r < issued; ++r)
                mbar_wait(&s_bar[r & 1], (((r & 1) ? ph1 : ph0) + (r >> 1)) & 1u);
        }
        ph0 += (issued + 1) >> 1;                        // rounds 0, 2, 4, ... used barrier 0
        ph1 += issued >> 1;
        return ok;
    };
    if constexpr (!PERSIST) {
        __syncthreads();                              // barriers initialised
        replay_tile(blockIdx.x);
    } else {
        for (;;) {
            __syncthreads();                              // the previous tile's shared reads are done
            if (threadIdx.x == 0) s_tile = (int)atomicAdd(work, 1u);
            __syncthreads();
            const int gt = s_tile;
            if (gt >= vt.total_tiles) return;
            if (!replay_tile(gt)) return;                 // a wait timed out: phases unknown, stop claiming
        }
    }
}

// add (r,g,b) to texel t of a [.][.][3] float array: texel t starts at float
// 3t, so (r,g) is 8-byte aligned for even t and (g,b) for odd t -- one
// vector and one scalar reduction
__device__ __forceinline__ void red_texel(float *d_tex, size_t t, float r, float g, float b) {
    float *d = d_tex + t * 3;
    if ((t & 1) == 0) {
        atomicAdd(reinterpret_cast<float2 *>(d), make_float2(r, g));
        atomicAdd(d + 2, b);
    } else {
        atomicAdd(d, r);
        atomicAdd(reinterpret_cast<float2 *>(d + 1), make_float2(g, b));
    }
}

// One CTA per screen tile.  Each pixel with a triangle contributes
// T * w_k * dL/dI_h to the 4 texels of its bilinear footprint.  The tile's
// taps fall in a small texel box when the tile lies on one chart: they are
// summed in shared memory (per-texel fixed point) and every touched texel is
// flushed with one global reduction; a tile whose box exceeds kTexCap texels
// (it straddles charts) reduces straight to global memory.
constexpr int kTexCap = 768;

// The bilinear footprint of one pixel: its four texels (clamped), weights and
// the T-weighted upstream gradient.
struct TexTaps {
    bool act;
    float g0, g1, g2, gm;        // gradient per channel, its largest magnitude
    int xa, xb, ya, yb;          // texel columns and rows
    float w[4];                  // weights of (xa,ya), (xb,ya), (xa,yb), (xb,yb)
};

// A thread owns two horizontally adjacent pixels of one row (x, x + 1), so
// the tile's box, scale and flush set-up is shared by them; where the
// texture is magnified they usually sample the same four texels, and their
// taps are then merged in registers before the shared-memory atomics
// (neighbouring pixels' atomics on one texel serialise).
template <int TW, int TH, int PX>
__global__ void __launch_bounds__(TW *TH / PX)
texture_bwd_kernel(ViewTable vt, const float *__restrict__ mesh_depth, const float *__restrict__ uv,
                   const float *__restrict__ out_T, const float *__restrict__ dL_drgb,
                   const float *__restrict__ dL_dmesh, int tw, int th, float *__restrict__ d_tex) {
    static_assert(PX == 2 && TW % 2 == 0, "pixel pairs along a row");
    constexpr int NT = TW * TH / 2;
    static_assert(NT % 32 == 0, "whole warps");
    // per texel: the fixed-point sums of the three channels (one plane each,
    // so a warp's consecutive texels fall in consecutive banks), then the
    // largest tap
    __shared__ int s_acc[kTexCap * 4];
    __shared__ int s_box[4];
    const int gt = blockIdx.x;
    const int v = view_of_tile(vt, gt);
    const ViewDev &V = vt.v[v];
    const int local = gt - V.tile_off;
    const int t = threadIdx.x;
    const int px0 = (local % V.tiles_x) * TW + (t % (TW / 2)) * 2;
    const int py = (local / V.tiles_x) * TH + t / (TW / 2);
    const long long npx = (long long)V.W * V.H;
    TexTaps tp[2];
    int mx0 = 0x7fffffff, mx1 = -1, my0 = 0x7fffffff, my1 = -1;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        TexTaps &a = tp[q];
        const int px = px0 + q;
        const bool inside = px < V.W && py < V.H;
        const long long lp = (long long)py * V.W + px;
        const long long gp = V.pix_off + lp;
        a.act = inside && mesh_depth[gp] < INFINITY;
        a.g0 = a.g1 = a.g2 = 0.f;
        float fx = 0.f, fy = 0.f;
        int ix = 0, iy = 0;
        if (a.act) {
            const float T = out_T[gp];
            const float *g = dL_drgb + 3 * V.pix_off + lp;
            a.g0 = T * g[0]; a.g1 = T * g[npx]; a.g2 = T * g[2 * npx];
            if (dL_dmesh) {   // a loss on the mesh colour itself (no T factor)
                const float *gm = dL_dmesh + 3 * V.pix_off + lp;
                a.g0 += gm[0]; a.g1 += gm[npx]; a.g2 += gm[2 * npx];
            }
            const float *u = uv + 2 * V.pix_off + lp;
            const float ss = u[0] * (float)tw - 0.5f, tt = u[npx] * (float)th - 0.5f;
            const float x0 = floorf(ss), y0 = floorf(tt);
            fx = ss - x0; fy = tt - y0;
            ix = (int)fmaxf(fminf(x0, 1e8f), -1e8f);
            iy = (int)fmaxf(fminf(y0, 1e8f), -1e8f);
        }
        a.gm = fmaxf(fabsf(a.g0), fmaxf(fabsf(a.g1), fabsf(a.g2)));
        a.xa = min(max(ix, 0), tw - 1); a.xb = min(max(ix + 1, 0), tw - 1);
        a.ya = min(max(iy, 0), th - 1); a.yb = min(max(iy + 1, 0), th - 1);
        a.w[0] = (1.f - fx) * (1.f - fy);
        a.w[1] = fx * (1.f - fy);
        a.w[2] = (1.f - fx) * fy;
        a.w[3] = fx * fy;
        if (a.act) {
            mx0 = min(mx0, a.xa); mx1 = max(mx1, a.xb);
            my0 = min(my0, a.ya); my1 = max(my1, a.yb);
        }
    }
    if (t == 0) {
        s_box[0] = 0x7fffffff; s_box[1] = -1; s_box[2] = 0x7fffffff; s_box[3] = -1;
    }
    __syncthreads();
    {
        mx0 = __reduce_min_sync(0xffffffffu, mx0);
        mx1 = __reduce_max_sync(0xffffffffu, mx1);
        my0 = __reduce_min_sync(0xffffffffu, my0);
        my1 = __reduce_max_sync(0xffffffffu, my1);
        if ((t & 31) == 0 && mx1 >= 0) {
            atomicMin(&s_box[0], mx0); atomicMax(&s_box[1], mx1);
            atomicMin(&s_box[2], my0); atomicMax(&s_box[3], my1);
        }
    }
    __syncthreads();
    const int bx0 = s_box[0], by0 = s_box[2];
    if (s_box[1] < 0) return;
    const int bw = s_box[1] - bx0 + 1, bh = s_box[3] - by0 + 1;
    // the pair's footprints coincide: one merged set of four taps
    const bool same = tp[0].act && tp[1].act && tp[0].xa == tp[1].xa && tp[0].xb == tp[1].xb &&
                      tp[0].ya == tp[1].ya && tp[0].yb == tp[1].yb;
    if ((long long)bw * bh > kTexCap) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const TexTaps &a = tp[q];
            if (!a.act) continue;
            const int xs[4] = {a.xa, a.xb, a.xa, a.xb}, ys[4] = {a.ya, a.ya, a.yb, a.yb};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (a.w[k] != 0.f)
                    red_texel(d_tex, (size_t)ys[k] * tw + xs[k], a.w[k] * a.g0, a.w[k] * a.g1, a.w[k] * a.g2);
        }
        return;
    }
    // Per-texel fixed point (native int32 shared atomics, exact and
    // order-independent sums).  Pass 1 takes, per texel, the largest tap
    // magnitude M over its three channels (the bits of a non-negative float
    // order like the float; a merged pair's tap counts as one).  Pass 2 adds
    // each tap in units of
    // 2^(e - 19), 2^e <= M < 2^(e+1): a tap is rounded to at most 2^-20 M, so
    // a texel's sums carry the rounding of its own taps whatever the tile's
    // other texels receive.  Every tap is at most M, a footprint's four taps
    // coincide only at a clamped corner and a tile holds at most 256
    // footprints, so |sum| <= 1024 M < 2^30 units.
    int *mx = s_acc + kTexCap * 3;
    const int ncell = bw * bh;
    for (int i = t; i < ncell; i += NT) {
        s_acc[i] = 0;
        s_acc[kTexCap + i] = 0;
        s_acc[2 * kTexCap + i] = 0;
        mx[i] = 0;
    }
    __syncthreads();
    // tap k of the thread's footprint(s): value per channel and its largest
    // magnitude (0 for a zero weight)
    auto taps = [&](int q, int k, float &v0, float &v1, float &v2, float &m) {
        if (same) {
            const float wa = tp[0].w[k], wb = tp[1].w[k];
            v0 = fmaf(wa, tp[0].g0, wb * tp[1].g0);
            v1 = fmaf(wa, tp[0].g1, wb * tp[1].g1);
            v2 = fmaf(wa, tp[0].g2, wb * tp[1].g2);
            m = fmaxf(fabsf(v0), fmaxf(fabsf(v1), fabsf(v2)));
        } else {
            const float w = tp[q].w[k];
            v0 = w * tp[q].g0; v1 = w * tp[q].g1; v2 = w * tp[q].g2;
            m = w * tp[q].gm;
        }
    };
    const int nq = same ? 1 : 2;
    for (int q = 0; q < nq; ++q) {
        if (!tp[q].act) continue;
        const int xs[4] = {tp[q].xa, tp[q].xb, tp[q].xa, tp[q].xb};
        const int ys[4] = {tp[q].ya, tp[q].ya, tp[q].yb, tp[q].yb};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float v0, v1, v2, m;
            taps(q, k, v0, v1, v2, m);
            if (m != 0.f) atomicMax(mx + (ys[k] - by0) * bw + (xs[k] - bx0), __float_as_int(m));
        }
    }
    __syncthreads();
    // 2^(19 - e) and 2^(e - 19) for the texel whose largest tap has exponent e
    auto unit_inv = [](int mbits) {
        const int e = ((mbits >> 23) & 0xff) - 127;
        return __int_as_float((min(max(19 - e, -126), 127) + 127) << 23);
    };
    auto unit = [](int mbits) {
        const int e = ((mbits >> 23) & 0xff) - 127;
        return __int_as_float((127 - min(max(19 - e, -126), 127)) << 23);
    };
    for (int q = 0; q < nq; ++q) {
        if (!tp[q].act) continue;
        const int xs[4] = {tp[q].xa, tp[q].xb, tp[q].xa, tp[q].xb};
        const int ys[4] = {tp[q].ya, tp[q].ya, tp[q].yb, tp[q].yb};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float v0, v1, v2, m;
            taps(q, k, v0, v1, v2, m);
            if (m == 0.f) continue;
            const int c = (ys[k] - by0) * bw + (xs[k] - bx0);
            const float ui = unit_inv(mx[c]);
            atomicAdd(s_acc + c, __float2int_rn(v0 * ui));
            atomicAdd(s_acc + kTexCap + c, __float2int_rn(v1 * ui));
            atomicAdd(s_acc + 2 * kTexCap + c, __float2int_rn(v2 * ui));
        }
    }
    __syncthreads();
    for (int i = t; i < ncell; i += NT) {
        const int r = s_acc[i], gg = s_acc[kTexCap + i], b = s_acc[2 * kTexCap + i];
        if (r != 0 || gg != 0 || b != 0) {
            const float u = unit(mx[i]);
            red_texel(d_tex, (size_t)(by0 + i / bw) * tw + (bx0 + i % bw), (float)r * u, (float)gg * u,
                      (float)b * u);
        }
    }
}

// The (Gaussian, view) pairs with a gradient: the records whose nine
// partials the replay left not all zero.  Only a few percent of the records
// of a 1080p view have tiles, so the chain rule below runs on a list of
// those pairs, not on every Gaussian: one thread per record reads its
// partials (consecutive records contiguous: coalesced) and appends
// (Gaussian, view), one atomic per warp.  A Gaussian no view blended has no
// gradient: nothing is added (this also keeps culled, non-finite parameters
// out of the chain rule).
__global__ void __launch_bounds__(256)
pbwd_scan_kernel(int n, long long n_rec, const float *__restrict__ g2d, uint2 *__restrict__ list,
                 unsigned int *__restrict__ count) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false;
    if (r < n_rec) {
        const float *gg = g2d + r * kG;
#pragma unroll
        for (int q = 0; q < kG; ++q) any |= gg[q] != 0.f;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, any);
    if (bal == 0u) return;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == __ffs(bal) - 1) base = atomicAdd(count, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
    if (any) {
        const int v = (int)(r / n);
        list[base + __popc(bal & lanemask_lt())] = make_uint2((uint32_t)(r - (long long)v * n), (uint32_t)v);
    }
}

template <int DEG, bool F16>
__global__ void __launch_bounds__(128, 4)
project_bwd_kernel(ViewTable vt, int n, const float *__restrict__ means,
                   const float *__restrict__ scales, const float *__restrict__ quats,
                   const float *__restrict__ opac, const void *__restrict__ sh_raw, Filters flt,
                   const float *__restrict__ g2d, const uint2 *__restrict__ list,
                   const unsigned int *__restrict__ count, float *__restrict__ d_means,
                   float *__restrict__ d_scales, float *__restrict__ d_quats,
                   float *__restrict__ d_opac, float *__restrict__ d_sh) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    // SH gradient accumulators, one private column per thread (conflict-free
    // [k][c][thread] layout): keeps 3K values out of the register file
    __shared__ float s_gsh[K * 3][128];
    // the cameras, for the lanes of a warp that walk different views at once
    __shared__ ViewDev s_view[HM_MAX_VIEWS];
    {
        const int words = vt.n_views * (int)(sizeof(ViewDev) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(vt.v);
        int *dst = reinterpret_cast<int *>(s_view);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    }
    auto one_gaussian = [&](const int i, const uint32_t vmask) {
        float(*gsh)[128] = s_gsh;
        const int tl = threadIdx.x;
        const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
        // Mip-Splatting's 3D filter: effective scales se_k = sqrt(s_k^2 + v) and
        // the opacity factor rho3 = prod_k s_k / se_k (v is a constant)
        const float v3 = flt.f3d ? flt.f3d[i] : 0.f;
        float se[3] = {s[0], s[1], s[2]}, rho3 = 1.f;
        if (v3 > 0.f) {
    #pragma unroll
            for (int k = 0; k < 3; ++k) {
                se[k] = sqrtf(fmaf(s[k], s[k], v3));
                rho3 *= s[k] / se[k];
            }
        }
        const float op_i = opac[i];
        float g_rho3 = 0.f;                 // dL/drho3 over the views
        const float4 q4 = reinterpret_cast<const float4 *>(quats)[i];
        const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
        const float qinv = rsqrtf(qn2);
        const float qw = q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
        const float R[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                               {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                               {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
        float M[3][3];
    #pragma unroll
        for (int a = 0; a < 3; ++a)
    #pragma unroll
            for (int k = 0; k < 3; ++k) M[a][k] = R[a][k] * se[k];
        // SH coefficients are re-read (L1-resident after the first view) where
        // they are used instead of being held across the view loop
        const __half *sh_h = reinterpret_cast<const __half *>(sh_raw) + (size_t)i * K * 3;
        const float *sh_f = reinterpret_cast<const float *>(sh_raw) + (size_t)i * K * 3;
        auto ld_sh = [&](int j) -> float { return F16 ? __half2float(sh_h[j]) : __ldg(sh_f + j); };
        float gmean[3] = {0.f, 0.f, 0.f};
        float gM[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    #pragma unroll
        for (int k = 0; k < K * 3; ++k) gsh[k][tl] = 0.f;
        float gop = 0.f;
        bool touched = false;           // some view blended it
        for (uint32_t m = vmask; m != 0u; m &= m - 1u) {
            const int v = __ffs(m) - 1;
            const float *gg = g2d + ((size_t)v * n + i) * kG;
            float g[kG];
    #pragma unroll
            for (int q = 0; q < kG; ++q) g[q] = gg[q];
            // the replay sums the moments of dL/dq / ln 2 (q = K d^2, alpha = o 2^q)
    #pragma unroll
            for (int q = 0; q < 5; ++q) g[q] *= kLn2;
            // a record with gradient was blended, so the forward kept it (its
            // FP64-rounded depth passed the near plane); the Jacobian only needs
            // the view position to FP32 accuracy, so it is recomputed in FP32
            // here (the FP64 pipe is ~1/64 of the FP32 rate)
            const ViewDev &V = s_view[v];
            const float zf = fmaf(V.R[6], mx, fmaf(V.R[7], my, fmaf(V.R[8], mz, V.t[2])));
            if (!(zf > 0.f)) continue;
            touched = true;
            const float txf = fmaf(V.R[0], mx, fmaf(V.R[1], my, fmaf(V.R[2], mz, V.t[0])));
            const float tyf = fmaf(V.R[3], mx, fmaf(V.R[4], my, fmaf(V.R[5], mz, V.t[1])));
            const float rz = __frcp_rn(zf);
            const float rx = txf * rz, ry = tyf * rz;
            const float limx = 1.3f * (0.5f * (float)V.W / V.fx), limy = 1.3f * (0.5f * (float)V.H / V.fy);
            const bool inx = rx > -limx && rx < limx, iny = ry > -limy && ry < limy;
            const float rxc = fminf(limx, fmaxf(-limx, rx)), ryc = fminf(limy, fmaxf(-limy, ry));
            const float J00 = V.fx * rz, J02 = -V.fx * rxc * rz, J11 = V.fy * rz, J12 = -V.fy * ryc * rz;
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
            const float h = flt.kernel;
            const float A0 = V0[0] * V0[0] + V0[1] * V0[1] + V0[2] * V0[2];
            const float C0 = V1[0] * V1[0] + V1[1] * V1[1] + V1[2] * V1[2];
            const float a = A0 + h, c = C0 + h;
            const float b = V0[0] * V1[0] + V0[1] * V1[1] + V0[2] * V1[2];
            const float cx_ = V0[1] * V1[2] - V0[2] * V1[1], cy_ = V0[2] * V1[0] - V0[0] * V1[2],
                        cz_ = V0[0] * V1[1] - V0[1] * V1[0];
            const float det0 = cx_ * cx_ + cy_ * cy_ + cz_ * cz_;      // det(Sigma2D)
            const float det = det0 + h * (A0 + C0) + h * h;
            const float rd2 = 1.f / (det * det);
            // the blend's moments S of dL/dq (q = K d^2): dL/dmean2d = -2K conic S_(dx,dy),
            // dL/dconic = K (S_dx2, 2 S_dxdy, S_dy2)
            const float rdet = 1.f / det;
            const float cxx = c * rdet, cxy = -b * rdet, cyy = a * rdet;
            const float gmx = -2.f * kConicScale * (cxx * g[0] + cxy * g[1]);
            const float gmy = -2.f * kConicScale * (cxy * g[0] + cyy * g[1]);
            // conic (c/det, -b/det, a/det) -> Sigma' entries
            const float gA = kConicScale * g[2], gB = 2.f * kConicScale * g[3], gC = kConicScale * g[4];
            float ga = (-c * c * gA + b * c * gB - b * b * gC) * rd2;
            float gb = (2.f * b * c * gA - (a * c + b * b) * gB + 2.f * a * b * gC) * rd2;
            float gc = (-b * b * gA + a * b * gB - a * a * gC) * rd2;
            // the record's opacity is op rho3 rho2; with the 2D Mip filter
            // rho2 = sqrt(D0 / D1), D0 = A0 C0 - b^2, D1 = (A0 + h)(C0 + h) - b^2, so
            // drho2 = rho2 / 2 (dD0 / D0 - dD1 / D1)
            float rho2 = 1.f;
            if (flt.antialias) {
                rho2 = det0 > 0.f ? sqrtf(det0 * rdet) : 0.f;
                if (det0 > 0.f) {
                    const float k2 = 0.5f * g[5] * op_i * rho3 * rho2, r0 = 1.f / det0;
                    ga += k2 * (C0 * r0 - c * rdet);
                    gc += k2 * (A0 * r0 - a * rdet);
                    gb += 2.f * k2 * b * (rdet - r0);
                }
            }
            g_rho3 += g[5] * op_i * rho2;
            // Sigma' = V V^T: dV0 = 2 ga V0 + gb V1, dV1 = gb V0 + 2 gc V1
            float gV0[3], gV1[3];
    #pragma unroll
            for (int k = 0; k < 3; ++k) {
                gV0[k] = 2.f * ga * V0[k] + gb * V1[k];
                gV1[k] = gb * V0[k] + 2.f * gc * V1[k];
            }
            // V = T M: dM += T^T dV, dT = dV M^T
            float gT0[3], gT1[3];
    #pragma unroll
            for (int r = 0; r < 3; ++r) {
    #pragma unroll
                for (int k = 0; k < 3; ++k) gM[r][k] += T0[r] * gV0[k] + T1[r] * gV1[k];
                gT0[r] = gV0[0] * M[r][0] + gV0[1] * M[r][1] + gV0[2] * M[r][2];
                gT1[r] = gV1[0] * M[r][0] + gV1[1] * M[r][1] + gV1[2] * M[r][2];
            }
            // T = J W (J01 = J10 = 0)
            float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f;
    #pragma unroll
            for (int k = 0; k < 3; ++k) {
                gJ00 += gT0[k] * V.R[k];
                gJ02 += gT0[k] * V.R[6 + k];
                gJ11 += gT1[k] * V.R[3 + k];
                gJ12 += gT1[k] * V.R[6 + k];
            }
            const float rz2 = rz * rz;
            float gtx = 0.f, gty = 0.f, gtz = 0.f;
            gtz += -gJ00 * V.fx * rz2 - gJ11 * V.fy * rz2;
            // J02 = -fx xc / z with xc = clamp(x/z)
            gtz += gJ02 * V.fx * rxc * rz2;
            gtz += gJ12 * V.fy * ryc * rz2;
            if (inx) {
                gtx += -gJ02 * V.fx * rz2;
                gtz += gJ02 * V.fx * rx * rz2;
            }
            if (iny) {
                gty += -gJ12 * V.fy * rz2;
                gtz += gJ12 * V.fy * ry * rz2;
            }
            // mean2d = (fx x/z + cx, fy y/z + cy)
            gtx += gmx * V.fx * rz;
            gty += gmy * V.fy * rz;
            gtz += -(gmx * V.fx * rx + gmy * V.fy * ry) * rz;
            // t = W mean + t_cam
    #pragma unroll
            for (int k = 0; k < 3; ++k) gmean[k] += V.R[k] * gtx + V.R[3 + k] * gty + V.R[6 + k] * gtz;
            gop += g[5] * rho3 * rho2;
            // colour
            float d0 = mx - V.campos[0], d1 = my - V.campos[1], d2 = mz - V.campos[2];
            const float dinv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            d0 *= dinv; d1 *= dinv; d2 *= dinv;
            float Y[K];
            sh_basis<DEG>(d0, d1, d2, Y);
            float gcol[3] = {g[6], g[7], g[8]};
    #pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float acc = 0.5f;
    #pragma unroll
                for (int k = 0; k < K; ++k) acc = fmaf(Y[k], ld_sh(3 * k + ch), acc);
                if (acc < 0.f) gcol[ch] = 0.f;   // clamped at 0: no gradient
    #pragma unroll
                for (int k = 0; k < K; ++k) gsh[3 * k + ch][tl] += Y[k] * gcol[ch];
            }
            if (DEG > 0) {
                float wk[K];
    #pragma unroll
                for (int k = 0; k < K; ++k)
                    wk[k] = ld_sh(3 * k) * gcol[0] + ld_sh(3 * k + 1) * gcol[1] + ld_sh(3 * k + 2) * gcol[2];
                float gd[3];
                sh_grad_dot<DEG>(d0, d1, d2, wk, gd[0], gd[1], gd[2]);
                const float dd = gd[0] * d0 + gd[1] * d1 + gd[2] * d2;
                gmean[0] += (gd[0] - dd * d0) * dinv;
                gmean[1] += (gd[1] - dd * d1) * dinv;
                gmean[2] += (gd[2] - dd * d2) * dinv;
            }
        }
        if (!touched) return;
        // M = R S: dS_k = sum_a dM[a][k] R[a][k], dR[a][k] = dM[a][k] s_k
        float gR[3][3];
        float gs[3] = {0.f, 0.f, 0.f};
    #pragma unroll
        for (int a = 0; a < 3; ++a)
    #pragma unroll
            for (int k = 0; k < 3; ++k) {
                gs[k] += gM[a][k] * R[a][k];
                gR[a][k] = gM[a][k] * se[k];
            }
        // through se_k = sqrt(s_k^2 + v) and rho3 = prod_j s_j / se_j:
        // dse_k/ds_k = s_k / se_k, drho3/ds_k = rho3 v / (s_k se_k^2)
        if (v3 > 0.f) {
    #pragma unroll
            for (int k = 0; k < 3; ++k) gs[k] = gs[k] * (s[k] / se[k]) + g_rho3 * rho3 * v3 / (s[k] * se[k] * se[k]);
        }
        // R(q^) -> q^ (w, x, y, z)
        float gqw = 2.f * (qz * (gR[1][0] - gR[0][1]) + qy * (gR[0][2] - gR[2][0]) + qx * (gR[2][1] - gR[1][2]));
        float gqx = 2.f * (qy * (gR[0][1] + gR[1][0]) + qz * (gR[0][2] + gR[2][0]) + qw * (gR[2][1] - gR[1][2])) -
                    4.f * qx * (gR[1][1] + gR[2][2]);
        float gqy = 2.f * (qx * (gR[0][1] + gR[1][0]) + qz * (gR[1][2] + gR[2][1]) + qw * (gR[0][2] - gR[2][0])) -
                    4.f * qy * (gR[0][0] + gR[2][2]);
        float gqz = 2.f * (qx * (gR[0][2] + gR[2][0]) + qy * (gR[1][2] + gR[2][1]) + qw * (gR[1][0] - gR[0][1])) -
                    4.f * qz * (gR[0][0] + gR[1][1]);
        // normalisation q^ = q / |q|
        const float dot = gqw * qw + gqx * qx + gqy * qy + gqz * qz;
        gqw = (gqw - dot * qw) * qinv;
        gqx = (gqx - dot * qx) * qinv;
        gqy = (gqy - dot * qy) * qinv;
        gqz = (gqz - dot * qz) * qinv;
    #pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicAdd(d_means + 3 * i + k, gmean[k]);
            atomicAdd(d_scales + 3 * i + k, gs[k]);
        }
        // several views of a Gaussian run in parallel: atomic additions
        // (four-float vector atomics where the rows are 16-byte aligned)
        if (((uintptr_t)d_quats & 15) == 0) {
            atomicAdd(reinterpret_cast<float4 *>(d_quats) + i, make_float4(gqw, gqx, gqy, gqz));
        } else {
            atomicAdd(d_quats + 4 * i, gqw);
            atomicAdd(d_quats + 4 * i + 1, gqx);
            atomicAdd(d_quats + 4 * i + 2, gqy);
            atomicAdd(d_quats + 4 * i + 3, gqz);
        }
        atomicAdd(d_opac + i, gop);
        float *ds = d_sh + (size_t)i * K * 3;
        if constexpr ((K * 3) % 4 == 0) {
            if (((uintptr_t)ds & 15) == 0) {
    #pragma unroll
                for (int j = 0; j < K * 3; j += 4)
                    atomicAdd(reinterpret_cast<float4 *>(ds + j),
                              make_float4(gsh[j][tl], gsh[j + 1][tl], gsh[j + 2][tl], gsh[j + 3][tl]));
                return;
            }
        }
    #pragma unroll
        for (int j = 0; j < K * 3; ++j) atomicAdd(ds + j, gsh[j][tl]);
    };
    __syncthreads();
    // one listed (Gaussian, view) pair per thread
    const unsigned cnt = *count;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const uint2 it = list[e];
        if (hm_check(it.x < (uint32_t)n && it.y < (uint32_t)vt.n_views)) one_gaussian((int)it.x, 1u << it.y);
    }
}

template <int DEG>
cudaError_t launch_pbwd(const ViewTable &vt, int n, const float *means, const float *scales,
                        const float *quats, const float *opac, const void *sh, bool f16, Filters flt,
                        const float *g2d, uint2 *list, unsigned int *count, float *dm, float *ds,
                        float *dq, float *dop, float *dsh, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const long long n_rec = (long long)vt.n_views * n;
    pbwd_scan_kernel<<<(unsigned)((n_rec + 255) / 256), 256, 0, s>>>(n, n_rec, g2d, list, count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // a resident grid: the list holds a few percent of the records
    long long g = ((long long)vt.n_views * n + 127) / 128;
    if (g > 148 * 4) g = 148 * 4;
    const dim3 grid((unsigned)g);
    if (f16)
        project_bwd_kernel<DEG, true><<<grid, 128, 0, s>>>(vt, n, means, scales, quats, opac, sh, flt, g2d, list,
                                                          count, dm, ds, dq, dop, dsh);
    else
        project_bwd_kernel<DEG, false><<<grid, 128, 0, s>>>(vt, n, means, scales, quats, opac, sh, flt, g2d, list,
                                                           count, dm, ds, dq, dop, dsh);
    return cudaGetLastError();
}

}  // namespace

}  // namespace hm

namespace hm {
namespace {

// resident CTAs of a kernel at a block size and dynamic shared memory, over
// all SMs (cached per device and batch; the batch sets the shared memory)
template <typename K>
int resident_ctas(K kernel, int threads, int smem, int slot) {
    static int cache[64][6][8] = {};
    static int cache_smem[64][6][8] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const int b = smem <= 2048 ? 0 : smem <= 8192 ? 1 : smem <= 16384 ? 2 : smem <= 32768 ? 3 : 4;
    int &c = cache[dev][slot][b];
    if (c == 0 || cache_smem[dev][slot][b] != smem) {
        int per_sm = 0, nsm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        c = per_sm * nsm;
        cache_smem[dev][slot][b] = smem;
    }
    return c;
}

}  // namespace
}  // namespace hm

using namespace hm;

// Workspace layout: the replay's partials (kG floats per record), 16 bytes of
// counters (the persistent launch's tile counter, the length of the pair
// list), the list of (Gaussian, view) pairs with a gradient, and 256 spare
// bytes.  The replay clears the partials and the tile counter.
namespace {
struct BwdWs {
    float *g2d;
    unsigned int *tiles, *count;
    uint2 *list;
    size_t clear_bytes;
};
size_t bwd_ws_layout(int32_t n_views, int32_t n, void *ws, BwdWs *w) {
    const size_t g2d_bytes = sizeof(float) * kG * (size_t)n_views * (size_t)n;
    const size_t ctr = (g2d_bytes + 15) & ~(size_t)15, lst = ctr + 16;
    if (w) {
        unsigned char *b = reinterpret_cast<unsigned char *>(ws);
        w->g2d = reinterpret_cast<float *>(b);
        w->tiles = reinterpret_cast<unsigned int *>(b + ctr);
        w->count = w->tiles + 1;
        w->list = reinterpret_cast<uint2 *>(b + lst);
        w->clear_bytes = ctr + sizeof(unsigned int);
    }
    return lst + sizeof(uint2) * (size_t)n_views * (size_t)n + 256;
}
}  // namespace

extern "C" size_t hm_blend_backward_workspace_size(int32_t n_views, int32_t n) {
    if (n_views < 1 || n < 0) return 0;
    return bwd_ws_layout(n_views, n, nullptr, nullptr);
}

extern "C" hm_status hm_blend_backward(const hm_camera *cams, int32_t n_views, int32_t n,
                                       const float *means, const float *scales, const float *quats,
                                       const float *opacity, const float *filter_3d, const void *sh,
                                       int32_t sh_degree, int32_t sh_format, const void *records,
                                       const uint32_t *pair_vals, const uint32_t *tile_ranges,
                                       const float *mesh_depth, const float *mesh_rgb,
                                       const float *mesh_uv, int32_t tex_w, int32_t tex_h,
                                       const hm_options *opt, const float *out_T,
                                       const uint32_t *last_idx, const float *dL_drgb,
                                       const float *dL_dT, const float *dL_dmesh, float *d_means,
                                       float *d_scales, float *d_quats, float *d_opacity, float *d_sh,
                                       float *d_tex, int32_t *d_status, void *ws, size_t ws_bytes,
                                       void *stream) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt)) return HM_ERR_INVALID_ARG;
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (sh_degree < 0 || sh_degree > 3) return fail(HM_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (sh_format != HM_SH_F32 && sh_format != HM_SH_F16) return fail(HM_ERR_INVALID_ARG, "sh_format");
    if (!(opt->kernel_2d >= 0.f && opt->kernel_2d < 1e6f)) return fail(HM_ERR_INVALID_ARG, "kernel_2d");
    if (opt->batch < 1 || opt->batch > opt->tile_w * opt->tile_h)
        return fail(HM_ERR_INVALID_ARG, "batch must be in 1..%d for this tile shape", opt->tile_w * opt->tile_h);
    if (!tile_ranges || !out_T || !last_idx || !dL_drgb) return fail(HM_ERR_INVALID_ARG, "null pointer");
    if (n > 0 && (!means || !scales || !quats || !opacity || !sh || !records || !pair_vals ||
                  !d_means || !d_scales || !d_quats || !d_opacity || !d_sh))
        return fail(HM_ERR_INVALID_ARG, "null pointer");
    if (d_tex && (!mesh_depth || !mesh_uv || tex_w <= 0 || tex_h <= 0))
        return fail(HM_ERR_INVALID_ARG, "texture gradient needs mesh_depth, mesh_uv and the texture size");
    if ((uintptr_t)d_tex & 7) return fail(HM_ERR_INVALID_ARG, "d_tex must be 8-byte aligned");
    if (((uintptr_t)records & 15) || ((uintptr_t)quats & 15))
        return fail(HM_ERR_INVALID_ARG, "records and quats must be 16-byte aligned");
    const size_t need = hm_blend_backward_workspace_size(n_views, n);
    if (n > 0 && (!ws || ws_bytes < need)) return fail(HM_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    const float *bg = opt->bg;
    const int stages = opt->bwd_stages ? opt->bwd_stages : (HM_BWD_TEXTURE | HM_BWD_BLEND | HM_BWD_PROJECT);
    const Filters flt{filter_3d, opt->kernel_2d, opt->antialias ? 1 : 0};
    if (d_tex && (stages & HM_BWD_TEXTURE)) {
        dim3 tg(vt.total_tiles);
#define HM_TBWD(TW, TH, PX) \
    texture_bwd_kernel<TW, TH, PX><<<tg, TW * TH / PX, 0, s>>>(vt, mesh_depth, mesh_uv, out_T, dL_drgb, dL_dmesh, \
                                                           tex_w, tex_h, d_tex)
        if (opt->tile_w == 16) HM_TBWD(16, 16, 2);
        else if (opt->tile_w == 32) HM_TBWD(32, 8, 2);
        else HM_TBWD(8, 8, 2);
#undef HM_TBWD
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    if (n == 0) return HM_OK;
    BwdWs w;
    bwd_ws_layout(n_views, n, ws, &w);
    float *g2d = w.g2d;
    const Record *rec = reinterpret_cast<const Record *>(records);
    if (stages & HM_BWD_BLEND) {
    // the partials and the persistent launch's tile counter start at 0
    unsigned int *wq = opt->persistent ? w.tiles : nullptr;
    e = cudaMemsetAsync(g2d, 0, wq ? w.clear_bytes : sizeof(float) * kG * (size_t)n_views * n, s);
    if (e != cudaSuccess) return cuda_status(e);
    const uint32_t n_rec = (uint32_t)((long long)n_views * n);
    const int bwd_batch = opt->batch < kBwdBatchMax ? opt->batch : kBwdBatchMax;
    const size_t bwd_smem = 2 * (size_t)bwd_batch * (sizeof(Record) + sizeof(uint32_t));
#define HM_BBWD(TW, TH, PP, SLOT)                                                                                \
    do {                                                                                                         \
        auto kern = wq ? (dL_dT ? blend_bwd_kernel<TW, TH, PP, true, true> : blend_bwd_kernel<TW, TH, PP, true, false>) \
                       : (dL_dT ? blend_bwd_kernel<TW, TH, PP, false, true> : blend_bwd_kernel<TW, TH, PP, false, false>); \
        int grid = vt.total_tiles;                                                                               \
        if (wq) {                                                                                                \
            grid = resident_ctas(kern, TW * TH / (2 * PP), (int)bwd_smem, 2 * SLOT + (dL_dT ? 1 : 0));           \
            if (grid <= 0) return fail(HM_ERR_CUDA, "occupancy query failed");                                  \
            grid = grid < vt.total_tiles ? grid : vt.total_tiles;                                                \
        }                                                                                                        \
        kern<<<grid, TW * TH / (2 * PP), bwd_smem, s>>>(                                                          \
            vt, rec, n_rec, pair_vals, tile_ranges, mesh_rgb, bg[0], bg[1], bg[2], out_T, last_idx, dL_drgb,    \
            dL_dT, bwd_batch, g2d, d_status, wq);                                                               \
    } while (0)
    if (vt.total_tiles > 0) {
        if (opt->tile_w == 16) HM_BBWD(16, 16, 2, 0);
        else if (opt->tile_w == 32) HM_BBWD(32, 8, 1, 1);
        else HM_BBWD(8, 8, 1, 2);
    }
#undef HM_BBWD
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    if (!(stages & HM_BWD_PROJECT)) return HM_OK;
    const bool f16 = sh_format == HM_SH_F16;
    switch (sh_degree) {
        case 0: e = launch_pbwd<0>(vt, n, means, scales, quats, opacity, sh, f16, flt, g2d, w.list, w.count, d_means, d_scales, d_quats, d_opacity, d_sh, s); break;
        case 1: e = launch_pbwd<1>(vt, n, means, scales, quats, opacity, sh, f16, flt, g2d, w.list, w.count, d_means, d_scales, d_quats, d_opacity, d_sh, s); break;
        case 2: e = launch_pbwd<2>(vt, n, means, scales, quats, opacity, sh, f16, flt, g2d, w.list, w.count, d_means, d_scales, d_quats, d_opacity, d_sh, s); break;
        default: e = launch_pbwd<3>(vt, n, means, scales, quats, opacity, sh, f16, flt, g2d, w.list, w.count, d_means, d_scales, d_quats, d_opacity, d_sh, s); break;
    }
    return cuda_status(e);
}

// ---------------------------------------------------------------------------
// hm_blend_backward_noalloc: the same pass with its scratch in a static device
// array, for callers that cannot allocate (see hm.h).
// ---------------------------------------------------------------------------
namespace hm {
namespace {

static __device__ __align__(256) unsigned char g_bwd_noalloc_scratch[HM_BWD_NOALLOC_BYTES];

// Device address of the array.  The address belongs to the current context
// (a cudaDeviceReset, or a library loaded under another context, moves it),
// so it is looked up again on every call outside a stream capture; a call
// under capture, where the lookup may not run, uses the address the last
// uncaptured call on this device found.
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};

hm_status noalloc_scratch(cudaStream_t stream, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return fail(HM_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cs);
    const bool capturing = e != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    if (e != cudaSuccess) (void)cudaGetLastError();      // the query's own error is not the call's
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!capturing) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bwd_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        g_noalloc_ptr[dev] = p;
    } else if (!g_noalloc_ptr[dev]) {
        return fail(HM_ERR_INVALID_ARG,
                    "hm_blend_backward_noalloc: the first call on device %d (after any context "
                    "reset) must come before a stream capture", dev);
    }
    *out = g_noalloc_ptr[dev];
    return HM_OK;
}

}  // namespace
}  // namespace hm

extern "C" hm_status hm_blend_backward_noalloc(
    const hm_camera *cams, int32_t n_views, int32_t n, const float *means, const float *scales,
    const float *quats, const float *opacity, const float *filter_3d, const void *sh, int32_t sh_degree,
    int32_t sh_format, const void *records, const uint32_t *pair_vals, const uint32_t *tile_ranges,
    const float *mesh_depth, const float *mesh_rgb, const float *mesh_uv, int32_t tex_w,
    int32_t tex_h, const hm_options *opt, const float *out_T, const uint32_t *last_idx,
    const float *dL_drgb, const float *dL_dT, const float *dL_dmesh, float *d_means, float *d_scales,
    float *d_quats, float *d_opacity, float *d_sh, float *d_tex, int32_t *d_status, void *stream) {
    if (n_views < 1 || n < 0) return fail(HM_ERR_INVALID_ARG, "bad n_views or n");
    const size_t need = hm_blend_backward_workspace_size(n_views, n);
    if (need > HM_BWD_NOALLOC_BYTES)
        return fail(HM_ERR_INVALID_ARG,
                    "n_views * n = %lld needs %zu bytes of scratch, above the %u-byte static array "
                    "of hm_blend_backward_noalloc; use hm_blend_backward with a workspace",
                    (long long)n_views * n, need, (unsigned)HM_BWD_NOALLOC_BYTES);
    void *ws = nullptr;
    const hm_status st = noalloc_scratch((cudaStream_t)stream, &ws);
    if (st != HM_OK) return st;
    return hm_blend_backward(cams, n_views, n, means, scales, quats, opacity, filter_3d, sh, sh_degree,
                             sh_format, records, pair_vals, tile_ranges, mesh_depth, mesh_rgb,
                             mesh_uv, tex_w, tex_h, opt, out_T, last_idx, dL_drgb, dL_dT, dL_dmesh,
                             d_means, d_scales, d_quats, d_opacity, d_sh, d_tex, d_status, ws,
                             HM_BWD_NOALLOC_BYTES, stream);
}

#ifdef HM_CHECKED
namespace hm {
HM_CHECKED_READER(blend_bwd)
}  // namespace hm
#endif
