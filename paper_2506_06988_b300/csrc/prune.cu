// prune.cu -- the mesh-pruning metrics of Sec. 3.3 / Algorithm 1 (stage 1)
// on the GPU: per triangle
//  * normal variation: per training view, the alpha_normal % covered pixels
//    with the highest total variation of a prior normal map mark the
//    triangle they see (pixel -> triangle from hm_rasterize_mesh);
//  * adjacent angle: the triangle's normal differs by more than angle_deg
//    from a triangle sharing an edge;
//  * area: the alpha_area % smallest triangles;
//  * small pieces: edge-connected components of the triangles no metric
//    removed, of fewer than alpha_group triangles.
// The metrics are keep masks combined with && (a triangle survives only if
// none removes it).  Every decision is reproducible bit for bit by a CPU
// restatement: normals and squared areas in FP64 without fused operations,
// normal-map variation in FP32 in a fixed order, ranks by (key, index) from
// an exact radix select, components labelled by their smallest index.
#include <math.h>
#include <stdint.h>

#include "hm_host.h"

namespace hm {

namespace {

constexpr uint8_t kFlagNormal = 1, kFlagAngle = 2, kFlagArea = 4, kFlagGroup = 8;

// a face normal (x, y, z) and its squared norm w, FP64
struct __align__(32) Nrm {
    double x, y, z, w;
};

// ---- per-face geometry -----------------------------------------------------

__global__ void __launch_bounds__(256)
face_geom_kernel(int nf, int nv, const float *__restrict__ verts, const int32_t *__restrict__ faces,
                 Nrm *__restrict__ nrm, unsigned long long *__restrict__ n2key, int32_t *bad) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) {
        atomicOr(bad, 1);
        nrm[f] = Nrm{0.0, 0.0, 0.0, 0.0};
        n2key[f] = 0ull;
        return;
    }
    // (v1 - v0) x (v2 - v0) in FP64, every operation rounded on its own
    const double ax = __dsub_rn((double)verts[3 * i1], (double)verts[3 * i0]);
    const double ay = __dsub_rn((double)verts[3 * i1 + 1], (double)verts[3 * i0 + 1]);
    const double az = __dsub_rn((double)verts[3 * i1 + 2], (double)verts[3 * i0 + 2]);
    const double bx = __dsub_rn((double)verts[3 * i2], (double)verts[3 * i0]);
    const double by = __dsub_rn((double)verts[3 * i2 + 1], (double)verts[3 * i0 + 1]);
    const double bz = __dsub_rn((double)verts[3 * i2 + 2], (double)verts[3 * i0 + 2]);
    const double cx = __dsub_rn(__dmul_rn(ay, bz), __dmul_rn(az, by));
    const double cy = __dsub_rn(__dmul_rn(az, bx), __dmul_rn(ax, bz));
    const double cz = __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
    const double n2 = __dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz));
    nrm[f] = Nrm{cx, cy, cz, n2};
    n2key[f] = (unsigned long long)__double_as_longlong(n2);     // n2 >= 0: bits order like values
}

// vertex -> incident faces (counting sort; the order within a vertex does not
// matter to any metric)
__global__ void __launch_bounds__(256)
vert_count_kernel(int nf, const int32_t *__restrict__ faces, const int32_t *bad, uint32_t *__restrict__ cnt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || *bad) return;
#pragma unroll
    for (int e = 0; e < 3; ++e) atomicAdd(&cnt[faces[3 * f + e]], 1u);
}

__global__ void __launch_bounds__(256)
vert_fill_kernel(int nf, const int32_t *__restrict__ faces, const int32_t *bad, uint32_t *__restrict__ cursor,
                 uint32_t *__restrict__ vface) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || *bad) return;
#pragma unroll
    for (int e = 0; e < 3; ++e) vface[atomicAdd(&cursor[faces[3 * f + e]], 1u)] = (uint32_t)f;
}

__device__ __forceinline__ bool has_vertex(const int32_t *faces, uint32_t g, int32_t b) {
    return faces[3 * g] == b || faces[3 * g + 1] == b || faces[3 * g + 2] == b;
}

// Adjacent-angle test: n_f . n_g < cos_t sqrt(|n_f|^2 |n_g|^2) for some g
// sharing an edge (zero-area faces take no part).  Symmetric, so each face
// decides its own flag.
__global__ void __launch_bounds__(256)
angle_kernel(int nf, const int32_t *__restrict__ faces, const Nrm *__restrict__ nrm,
             const uint32_t *__restrict__ voff, const uint32_t *__restrict__ vcnt,
             const uint32_t *__restrict__ vface, double cos_t, const int32_t *bad, uint8_t *__restrict__ flags) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || *bad) return;
    const Nrm a = nrm[f];
    if (!(a.w > 0.0)) return;
    bool sharp = false;
    for (int e = 0; e < 3 && !sharp; ++e) {
        const int32_t va = faces[3 * f + e], vb = faces[3 * f + (e + 1) % 3];
        const uint32_t o = voff[va], c = vcnt[va];
        for (uint32_t k = 0; k < c; ++k) {
            const uint32_t g = vface[o + k];
            if (g == (uint32_t)f || !has_vertex(faces, g, vb)) continue;
            const Nrm b = nrm[g];
            if (!(b.w > 0.0)) continue;
            const double dot = __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
            if (dot < __dmul_rn(cos_t, __dsqrt_rn(__dmul_rn(a.w, b.w)))) {
                sharp = true;
                break;
            }
        }
    }
    if (sharp) flags[f] |= kFlagAngle;
}

// ---- exact k-th smallest key by radix select ------------------------------
// The target is the element of rank `rank` (0-based) in (key, index) order
// among the candidates.  Each pass histograms one 8-bit digit of the
// candidates whose higher digits equal the prefix chosen so far; the pick
// step descends into the digit holding the target.  At the end `prefix` is
// the target key and `rank` its position among the equal keys.

struct SelState {
    unsigned long long prefix, mask;
    long long rank;     // target position among the remaining candidates
    int active;         // 0: nothing to select (k == 0)
};

template <class Key>
__global__ void __launch_bounds__(256)
sel_hist_kernel(long long n, const Key *__restrict__ keys, const int32_t *__restrict__ valid,
                const SelState *st, int shift, unsigned int *__restrict__ hist) {
    __shared__ unsigned int s_h[256];
    s_h[threadIdx.x] = 0u;
    __syncthreads();
    if (st->active) {
        const unsigned long long prefix = st->prefix, mask = st->mask;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            if (valid && valid[i] < 0) continue;
            const unsigned long long k = (unsigned long long)keys[i];
            if ((k & mask) != prefix) continue;
            atomicAdd(&s_h[(k >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    if (s_h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_h[threadIdx.x]);
}

// one CTA of 256 threads: thread b holds bin b; an exclusive scan of the
// counts finds the bin holding the target rank; the histogram is cleared
// for the next pass
__global__ void __launch_bounds__(256) sel_pick_kernel(SelState *st, unsigned int *hist, int shift) {
    __shared__ unsigned long long s_w[8];
    const int b = threadIdx.x, lane = b & 31, w = b >> 5;
    const int active = st->active;      // read by every thread before the one owner writes
    const long long r = st->rank;
    const unsigned long long h = hist[b];
    unsigned long long x = h;           // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    unsigned long long before = x - h;
    for (int k = 0; k < w; ++k) before += s_w[k];
    if (active) {
        if (r >= (long long)before && r < (long long)(before + h)) {
            st->rank = r - (long long)before;
            st->prefix |= (unsigned long long)b << shift;
            st->mask |= 255ull << shift;
        } else if (b == 255 && r >= (long long)(before + h)) {
            st->active = 0;   // fewer candidates than the rank (cannot happen for k <= count)
        }
    }
    hist[b] = 0u;
}

// k = floor(alpha * count / 100) -> the target rank k - 1
__global__ void sel_init_kernel(SelState *st, const unsigned long long *count, long long count_host,
                                double alpha) {
    const long long c = count ? (long long)*count : count_host;
    const long long k = (long long)floor(alpha * (double)c / 100.0);
    st->prefix = 0ull;
    st->mask = 0ull;
    st->rank = k - 1;
    st->active = k > 0 ? 1 : 0;
}

// equal-key flags for the index-ordered tie break
template <class Key>
__global__ void __launch_bounds__(256)
sel_eq_kernel(long long n, const Key *__restrict__ keys, const int32_t *__restrict__ valid, const SelState *st,
              uint32_t *__restrict__ eq) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool ok = st->active && !(valid && valid[i] < 0);
    eq[i] = ok && (unsigned long long)keys[i] == st->prefix ? 1u : 0u;
}

// the k selected: key < target, or key == target among the first rank + 1 equal ones
__device__ __forceinline__ bool selected(unsigned long long k, uint32_t eq_idx, const SelState &st) {
    return k < st.prefix || (k == st.prefix && (long long)eq_idx <= st.rank);
}

__global__ void __launch_bounds__(256)
area_mark_kernel(int nf, const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ eq_idx,
                 const SelState *st, uint8_t *__restrict__ flags) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || !st->active) return;
    if (selected(keys[f], eq_idx[f], *st)) flags[f] |= kFlagArea;
}

// ---- normal-map total variation ---------------------------------------------

// key = ~bits(TV) so that ascending keys are TV descending; TV in FP32:
// sum over channels of (|N(x+1,y) - N(x,y)| + |N(x,y+1) - N(x,y)|)
__global__ void __launch_bounds__(256)
tv_key_kernel(int W, int H, const float *__restrict__ nm, const int32_t *__restrict__ tri,
              uint32_t *__restrict__ key, unsigned long long *covered) {
    const long long np = (long long)W * H;
    unsigned int c = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p - (long long)y * W);
        float tv = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float *n = nm + ch * np;
            const float v = n[p];
            const float dx = x + 1 < W ? fabsf(__fsub_rn(n[p + 1], v)) : 0.f;
            const float dy = y + 1 < H ? fabsf(__fsub_rn(n[p + W], v)) : 0.f;
            tv = __fadd_rn(tv, __fadd_rn(dx, dy));
        }
        key[p] = ~__float_as_uint(tv);
        c += tri[p] >= 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(covered, (unsigned long long)c);
}

// a selected pixel marks its triangle (every writer stores the same 1)
__global__ void __launch_bounds__(256)
tv_mark_kernel(long long np, int nf, const uint32_t *__restrict__ key, const int32_t *__restrict__ tri,
               const uint32_t *__restrict__ eq_idx, const SelState *st, int32_t *bad, uint32_t *__restrict__ mark) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np || !st->active) return;
    const int32_t f = tri[p];
    if (f < 0) return;
    if (f >= nf) {
        atomicOr(bad, 2);
        return;
    }
    if (selected(key[p], eq_idx[p], *st)) mark[f] = 1u;
}

__global__ void __launch_bounds__(256)
mark_merge_kernel(int nf, const uint32_t *__restrict__ mark, uint8_t *__restrict__ flags) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < nf && mark[f]) flags[f] |= kFlagNormal;
}

// ---- small pieces (min-label union-find over shared edges) ------------------

__device__ __forceinline__ int32_t find_root(int32_t *parent, int32_t x) {
    int32_t p = parent[x];
    while (p != x) {
        x = p;
        p = parent[x];
    }
    return x;
}

__global__ void __launch_bounds__(256)
uf_init_kernel(int nf, const uint8_t *__restrict__ flags, int32_t *__restrict__ parent, uint32_t *__restrict__ cnt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    parent[f] = flags[f] ? -1 : f;
    cnt[f] = 0u;
}

__global__ void __launch_bounds__(256)
uf_hook_kernel(int nf, const int32_t *__restrict__ faces, const uint32_t *__restrict__ voff,
               const uint32_t *__restrict__ vcnt, const uint32_t *__restrict__ vface, int32_t *parent,
               int32_t *changed) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || parent[f] < 0) return;
    for (int e = 0; e < 3; ++e) {
        const int32_t va = faces[3 * f + e], vb = faces[3 * f + (e + 1) % 3];
        const uint32_t o = voff[va], c = vcnt[va];
        for (uint32_t k = 0; k < c; ++k) {
            const uint32_t g = vface[o + k];
            if (g <= (uint32_t)f || parent[g] < 0 || !has_vertex(faces, g, vb)) continue;
            const int32_t r1 = find_root(parent, f), r2 = find_root(parent, (int32_t)g);
            if (r1 == r2) continue;
            const int32_t lo = min(r1, r2), hi = max(r1, r2);
            // a union was needed: another round runs even if a concurrent
            // hook already lowered parent[hi] below lo (then lo and that
            // parent are joined in the next round)
            atomicMin(&parent[hi], lo);
            *changed = 1;
        }
    }
}

__global__ void __launch_bounds__(256)
uf_compress_kernel(int nf, int32_t *parent) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || parent[f] < 0) return;
    parent[f] = find_root(parent, f);
}

__global__ void __launch_bounds__(256)
uf_count_kernel(int nf, const int32_t *__restrict__ parent, uint32_t *__restrict__ cnt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || parent[f] < 0) return;
    atomicAdd(&cnt[parent[f]], 1u);
}

__global__ void __launch_bounds__(256)
uf_flag_kernel(int nf, const int32_t *__restrict__ parent, const uint32_t *__restrict__ cnt, int alpha_group,
               uint8_t *__restrict__ flags, int32_t *__restrict__ label) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int32_t r = parent[f];
    if (label) label[f] = r;
    if (r >= 0 && (long long)cnt[r] < (long long)alpha_group) flags[f] |= kFlagGroup;
}

int blocks(long long n) { return (int)((n + 255) / 256); }

struct PruneWs {
    Nrm *nrm;
    unsigned long long *n2key, *covered;
    uint32_t *vcnt, *voff, *vcur, *vface, *eq, *eq_idx, *tvkey, *cnt, *nmark;
    unsigned int *hist;
    int32_t *parent, *flags_dev;   // flags_dev[0]: bad input bits, [1]: changed
    SelState *sel;
    ScanWs scan;
};

PruneWs carve_prune(void *ws, long long nv, long long nf, long long max_pix, size_t *bytes) {
    WsCarver c(ws);
    PruneWs w;
    const long long m = nf > max_pix ? nf : max_pix;
    w.nrm = c.take<Nrm>(nf);
    w.n2key = c.take<unsigned long long>(nf);
    w.covered = c.take<unsigned long long>(1);
    w.vcnt = c.take<uint32_t>(nv);
    w.voff = c.take<uint32_t>(nv);
    w.vcur = c.take<uint32_t>(nv);
    w.vface = c.take<uint32_t>(3 * nf);
    w.eq = c.take<uint32_t>(m);
    w.eq_idx = c.take<uint32_t>(m);
    w.tvkey = c.take<uint32_t>(max_pix);
    w.cnt = c.take<uint32_t>(nf);
    w.nmark = c.take<uint32_t>(nf);
    w.hist = c.take<unsigned int>(256);
    w.parent = c.take<int32_t>(nf);
    w.flags_dev = c.take<int32_t>(2);
    w.sel = c.take<SelState>(1);
    const long long sn = nv > m ? nv : m;
    w.scan.tile_status = c.take<unsigned long long>(scan_tiles(sn) + 1);
    w.scan.ticket = c.take<unsigned int>(1);
    *bytes = c.off + 256;
    return w;
}

// rank selection over n keys of one kind, then the equal-key scan
template <class Key>
cudaError_t run_select(const Key *keys, long long n, const int32_t *valid, int n_bits, PruneWs &w,
                       cudaStream_t s) {
    cudaError_t e;
    const int g = (int)(blocks(n) < 148 * 8 ? blocks(n) : 148 * 8);
    for (int shift = n_bits - 8; shift >= 0; shift -= 8) {
        sel_hist_kernel<Key><<<g, 256, 0, s>>>(n, keys, valid, w.sel, shift, w.hist);
        sel_pick_kernel<<<1, 256, 0, s>>>(w.sel, w.hist, shift);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sel_eq_kernel<Key><<<blocks(n), 256, 0, s>>>(n, keys, valid, w.sel, w.eq);
    return launch_scan(w.eq, nullptr, w.eq_idx, n, nullptr, -1, nullptr, w.scan, s);
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" void hm_default_prune_params(hm_prune_params *p) {
    if (!p) return;
    p->alpha_normal = 20.f;
    p->alpha_area = 50.f;
    p->angle_deg = 45.f;
    p->alpha_group = 100;
}

static long long max_view_pixels(const hm_camera *cams, int32_t n_views) {
    long long m = 0;
    for (int v = 0; v < n_views; ++v) {
        const long long p = (long long)cams[v].width * cams[v].height;
        if (p > m) m = p;
    }
    return m;
}

extern "C" size_t hm_mesh_prune_workspace_size(const hm_camera *cams, int32_t n_views, int32_t n_verts,
                                               int32_t n_faces) {
    if (n_verts < 0 || n_faces < 0 || n_views < 0 || (n_views > 0 && !cams)) return 0;
    size_t bytes = 0;
    carve_prune(nullptr, n_verts, n_faces, n_views > 0 ? max_view_pixels(cams, n_views) : 0, &bytes);
    return bytes;
}

extern "C" hm_status hm_mesh_prune(const hm_camera *cams, int32_t n_views, const float *verts, int32_t n_verts,
                                   const int32_t *faces, int32_t n_faces, const int32_t *tri_id,
                                   const float *normals, const hm_prune_params *p, uint8_t *flags,
                                   int32_t *label, void *ws, size_t ws_bytes, void *stream) {
    if (!p || n_verts < 0 || n_faces < 0 || n_views < 0) return fail(HM_ERR_INVALID_ARG, "bad sizes or params");
    if (!(p->alpha_normal >= 0.f && p->alpha_normal <= 100.f) || !(p->alpha_area >= 0.f && p->alpha_area <= 100.f) ||
        !(p->angle_deg >= 0.f && p->angle_deg <= 180.f) || p->alpha_group < 0)
        return fail(HM_ERR_INVALID_ARG, "prune parameters out of range");
    const bool use_normal = n_views > 0 && tri_id && normals;
    if (n_views > 0 && !cams) return fail(HM_ERR_INVALID_ARG, "null cams");
    if (use_normal) {
        hm_options o;
        hm_default_options(&o);
        ViewTable vt;
        if (!build_view_table(cams, n_views, &o, &vt)) return HM_ERR_INVALID_ARG;
    }
    if (n_faces == 0) return HM_OK;
    if (!verts || !faces || !flags) return fail(HM_ERR_INVALID_ARG, "null pointer");
    const long long max_pix = use_normal ? max_view_pixels(cams, n_views) : 0;
    size_t need = 0;
    carve_prune(nullptr, n_verts, n_faces, max_pix, &need);
    if (!ws || ws_bytes < need) return fail(HM_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    PruneWs w = carve_prune(ws, n_verts, n_faces, max_pix, &need);
    const int nf = n_faces;
    cudaError_t e;
    if ((e = cudaMemsetAsync(flags, 0, (size_t)nf, s)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(w.flags_dev, 0, 2 * sizeof(int32_t), s)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(w.vcnt, 0, sizeof(uint32_t) * (size_t)n_verts, s)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(w.hist, 0, 256 * sizeof(unsigned int), s)) != cudaSuccess) return cuda_status(e);
    // geometry, incidence, angles
    face_geom_kernel<<<blocks(nf), 256, 0, s>>>(nf, n_verts, verts, faces, w.nrm, w.n2key, w.flags_dev);
    int32_t host_flags[2] = {0, 0};
    if ((e = cudaMemcpyAsync(host_flags, w.flags_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_status(e);
    if (host_flags[0] & 1) return fail(HM_ERR_INVALID_ARG, "a face index is out of range");
    vert_count_kernel<<<blocks(nf), 256, 0, s>>>(nf, faces, w.flags_dev, w.vcnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    if ((e = launch_scan(w.vcnt, nullptr, w.voff, n_verts, nullptr, -1, nullptr, w.scan, s)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(w.vcur, w.voff, sizeof(uint32_t) * (size_t)n_verts, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return cuda_status(e);
    vert_fill_kernel<<<blocks(nf), 256, 0, s>>>(nf, faces, w.flags_dev, w.vcur, w.vface);
    const double cos_t = cos((double)p->angle_deg * (3.14159265358979323846 / 180.0));
    angle_kernel<<<blocks(nf), 256, 0, s>>>(nf, faces, w.nrm, w.voff, w.vcnt, w.vface, cos_t, w.flags_dev, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    // the smallest areas
    sel_init_kernel<<<1, 1, 0, s>>>(w.sel, nullptr, nf, (double)p->alpha_area);
    if ((e = run_select<unsigned long long>(w.n2key, nf, nullptr, 64, w, s)) != cudaSuccess) return cuda_status(e);
    area_mark_kernel<<<blocks(nf), 256, 0, s>>>(nf, w.n2key, w.eq_idx, w.sel, flags);
    // normal variation, view by view
    if (use_normal) {
        if ((e = cudaMemsetAsync(w.nmark, 0, sizeof(uint32_t) * (size_t)nf, s)) != cudaSuccess) return cuda_status(e);
        long long pix_off = 0;
        for (int v = 0; v < n_views; ++v) {
            const int W = cams[v].width, H = cams[v].height;
            const long long np = (long long)W * H;
            const int32_t *tri = tri_id + pix_off;
            if ((e = cudaMemsetAsync(w.covered, 0, sizeof(unsigned long long), s)) != cudaSuccess) return cuda_status(e);
            tv_key_kernel<<<(int)(blocks(np) < 148 * 8 ? blocks(np) : 148 * 8), 256, 0, s>>>(
                W, H, normals + 3 * pix_off, tri, w.tvkey, w.covered);
            sel_init_kernel<<<1, 1, 0, s>>>(w.sel, w.covered, 0, (double)p->alpha_normal);
            if ((e = run_select<uint32_t>(w.tvkey, np, tri, 32, w, s)) != cudaSuccess) return cuda_status(e);
            tv_mark_kernel<<<blocks(np), 256, 0, s>>>(np, nf, w.tvkey, tri, w.eq_idx, w.sel, w.flags_dev, w.nmark);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
            pix_off += np;
        }
        mark_merge_kernel<<<blocks(nf), 256, 0, s>>>(nf, w.nmark, flags);
    }
    // small pieces of what the metrics kept
    uf_init_kernel<<<blocks(nf), 256, 0, s>>>(nf, flags, w.parent, w.cnt);
    for (int it = 0; it < 64; ++it) {
        if ((e = cudaMemsetAsync(w.flags_dev + 1, 0, sizeof(int32_t), s)) != cudaSuccess) return cuda_status(e);
        uf_hook_kernel<<<blocks(nf), 256, 0, s>>>(nf, faces, w.voff, w.vcnt, w.vface, w.parent, w.flags_dev + 1);
        uf_compress_kernel<<<blocks(nf), 256, 0, s>>>(nf, w.parent);
        if ((e = cudaMemcpyAsync(host_flags, w.flags_dev, sizeof(host_flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_status(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_status(e);
        if (!host_flags[1]) break;
    }
    if (host_flags[1]) return fail(HM_ERR_CUDA, "component labels did not converge in 64 rounds");
    uf_count_kernel<<<blocks(nf), 256, 0, s>>>(nf, w.parent, w.cnt);
    uf_flag_kernel<<<blocks(nf), 256, 0, s>>>(nf, w.parent, w.cnt, p->alpha_group, flags, label);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemcpyAsync(host_flags, w.flags_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_status(e);
    if (host_flags[0] & 2) return fail(HM_ERR_INVALID_ARG, "a tri_id is out of range");
    return HM_OK;
}
