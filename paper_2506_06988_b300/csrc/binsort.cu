// binsort.cu -- tile binning and the (tile, depth) sort of (Gaussian, tile)
// pairs (the "tile-wise sorting" of the splatting rasteriser, Sec. 1).
//
// The sort is an LSD radix sort of the key (tile << 32 | depth bits), done
// in two stages:
//  1. the four depth digits are sorted on the un-duplicated records (every
//     copy of a record carries the same depth, so sorting before duplication
//     gives the same order and touches V*N elements instead of P pairs);
//  2. pairs are emitted in that depth order and the tile digits are sorted
//     stably on the P pairs.
// Equal depths keep the record order (camera, then Gaussian index), so each
// tile's list is ordered by (FP32 depth, Gaussian index).
//
// Pairs are culled where the tile's farthest mesh depth is at or in front of
// the Gaussian (depth >= tile_max_depth): every pixel of the tile then stops
// before reaching it, so the pair cannot contribute (Sec. 3.4: only
// D_gs < D_m is blended).
#include "hm_host.h"

namespace hm {

namespace {

// d^2 along one edge of the rectangle: the edge's coordinate is fixed at e,
// the other coordinate f ranges over [lo, hi]; d^2 = p e^2 + 2 q e f + r f^2
// is minimised at f = -q e / r (clamped), rr = 1 / r
__device__ __forceinline__ float edge_min(float p, float q, float r, float rr, float e, float lo,
                                          float hi) {
    const float f = fminf(hi, fmaxf(lo, -q * e * rr));
    return fmaf(p * e, e, fmaf(2.f * q * e, f, r * f * f));
}

// A projected record as the binning needs it.
struct BinRec {
    float mx, my, a, b, c, ra, rc, depth;   // mean, conic, 1/conic_xx, 1/conic_yy, depth key
    int x0, x1, y0, y1, v;                  // tile rectangle, camera
};

__device__ __forceinline__ BinRec load_bin_rec(const Record *rec, long long it, int n) {
    BinRec r;
    const float4 A = rec[it].a, B = rec[it].b, C = rec[it].c;
    // undo the record's K scaling (one rounding each, far inside the
    // ellipse test's 0.2% slack)
    r.mx = A.x; r.my = A.y;
    r.a = A.z * (1.f / kConicScale);
    r.b = A.w * (0.5f / kConicScale);
    r.c = B.x * (1.f / kConicScale);
    r.ra = 1.f / r.a; r.rc = 1.f / r.c;
    r.depth = B.z;
    unpack_range(__float_as_uint(B.w), r.x0, r.x1);
    unpack_range(__float_as_uint(C.w), r.y0, r.y1);
    r.v = (int)(it / n);
    return r;
}

__device__ __forceinline__ int rec_tiles(const BinRec &r) {
    return (r.x0 <= r.x1 && r.y0 <= r.y1) ? (r.x1 - r.x0 + 1) * (r.y1 - r.y0 + 1) : 0;
}

__device__ __forceinline__ BinRec shfl_rec(const BinRec &r, int src) {
    BinRec o;
    o.mx = __shfl_sync(0xffffffffu, r.mx, src); o.my = __shfl_sync(0xffffffffu, r.my, src);
    o.a = __shfl_sync(0xffffffffu, r.a, src); o.b = __shfl_sync(0xffffffffu, r.b, src);
    o.c = __shfl_sync(0xffffffffu, r.c, src); o.ra = __shfl_sync(0xffffffffu, r.ra, src);
    o.rc = __shfl_sync(0xffffffffu, r.rc, src); o.depth = __shfl_sync(0xffffffffu, r.depth, src);
    o.x0 = __shfl_sync(0xffffffffu, r.x0, src); o.x1 = __shfl_sync(0xffffffffu, r.x1, src);
    o.y0 = __shfl_sync(0xffffffffu, r.y0, src); o.y1 = __shfl_sync(0xffffffffu, r.y1, src);
    o.v = __shfl_sync(0xffffffffu, r.v, src);
    return o;
}

// Is the pair (record, tile) kept?  Mesh cull: the tile's farthest mesh depth
// must lie behind the record (Sec. 3.4 blends only D_gs < D_m).  Ellipse
// test: the 3-sigma ellipse must reach the rectangle of the tile's in-image
// pixel centres -- the minimum of the convex d^2 over the rectangle is 0 with
// the mean inside, else on an edge; 9 is inflated by 0.2% so the test stays
// a superset of the blend's FP32 per-pixel test.
__device__ __forceinline__ bool keep_tile(const ViewTable &vt, const float *tmax, int ellipse,
                                          const BinRec &r, int tx, int ty) {
    const ViewDev &V = vt.v[r.v];
    if (tmax != nullptr && !(r.depth < tmax[V.tile_off + ty * V.tiles_x + tx])) return false;
    if (!ellipse) return true;
    const float x0 = (float)(tx * vt.tile_w) + 0.5f - r.mx;
    const float x1 = (float)(min((tx + 1) * vt.tile_w, V.W) - 1) + 0.5f - r.mx;
    const float y0 = (float)(ty * vt.tile_h) + 0.5f - r.my;
    const float y1 = (float)(min((ty + 1) * vt.tile_h, V.H) - 1) + 0.5f - r.my;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
    float m = fminf(edge_min(r.a, r.b, r.c, r.rc, x0, y0, y1), edge_min(r.a, r.b, r.c, r.rc, x1, y0, y1));
    m = fminf(m, fminf(edge_min(r.c, r.b, r.a, r.ra, y0, x0, x1), edge_min(r.c, r.b, r.a, r.ra, y1, x0, x1)));
    return m <= 9.0f * 1.002f;
}

// records with more tiles than this are binned by the whole warp
constexpr int kSmallRect = 8;

// per record: number of kept tiles and a visibility flag.  Small rectangles
// are walked by their own thread; large ones by the whole warp, one record
// at a time, lanes over tiles.
__global__ void __launch_bounds__(256)
bin_count_kernel(ViewTable vt, int n, const Record *__restrict__ rec, const float *__restrict__ tmax,
                 int ellipse, uint32_t *__restrict__ cnt, uint32_t *__restrict__ flag) {
    const long long m = (long long)vt.n_views * n;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // lane l of warp w takes element w + nw (l + 32 k): a warp's records are
    // spread over the whole range, so large ones do not pile up in one warp
    for (long long base = w0; base < m; base += nw * 32) {
        const long long it = base + (long long)lane * nw;
        const bool valid = it < m;
        BinRec r;
        int nt = 0;
        if (valid) {
            r = load_bin_rec(rec, it, n);
            nt = rec_tiles(r);
        } else {
            r = BinRec{};
        }
        uint32_t k = 0;
        if (nt > 0 && nt <= kSmallRect) {
            for (int ty = r.y0; ty <= r.y1; ++ty)
                for (int tx = r.x0; tx <= r.x1; ++tx) k += keep_tile(vt, tmax, ellipse, r, tx, ty);
        }
        unsigned big = __ballot_sync(0xffffffffu, nt > kSmallRect);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const BinRec q = shfl_rec(r, src);
            const int nx = q.x1 - q.x0 + 1, ntot = nx * (q.y1 - q.y0 + 1);
            uint32_t c = 0;
            for (int t0 = 0; t0 < ntot; t0 += 32) {
                const int t = t0 + lane;
                const bool kept = t < ntot && keep_tile(vt, tmax, ellipse, q, q.x0 + t % nx, q.y0 + t / nx);
                c += __popc(__ballot_sync(0xffffffffu, kept));
            }
            if (lane == src) k = c;
        }
        if (valid) {
            cnt[it] = k;
            flag[it] = k != 0;
        }
    }
}

// visible records, compacted in record order: depth-sort keys and record ids
__global__ void __launch_bounds__(256)
bin_compact_kernel(long long m, const Record *__restrict__ rec, const uint32_t *__restrict__ cnt,
                   const uint32_t *__restrict__ pos, uint32_t *__restrict__ dkey,
                   uint32_t *__restrict__ ditem) {
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < m;
         it += (long long)gridDim.x * blockDim.x) {
        if (cnt[it] == 0) continue;
        const uint32_t o = pos[it];
        dkey[o] = __float_as_uint(rec[it].b.z);
        ditem[o] = (uint32_t)it;
    }
}

// per depth-sorted visible record: write its kept (tile, record) pairs at its
// scan offset; same small/large split as the count
__global__ void __launch_bounds__(256)
bin_emit_kernel(ViewTable vt, int n, const Record *__restrict__ rec, const float *__restrict__ tmax,
                int ellipse, const uint32_t *__restrict__ sorted_items, const long long *n_vis,
                const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ offs,
                long long capacity, uint32_t *__restrict__ pkey, uint32_t *__restrict__ pval) {
    const long long m = *n_vis;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // strided as in the count: the depth order puts the large near-camera
    // records together, and a warp walks its large records one at a time
    for (long long base = w0; base < m; base += nw * 32) {
        const long long j = base + (long long)lane * nw;
        bool valid = j < m;
        uint32_t it = 0, k = 0;
        long long o = 0;
        BinRec r = BinRec{};
        int nt = 0;
        if (valid) {
            it = sorted_items[j];
            k = cnt[it];
            o = offs[j];
            valid = k > 0 && o + k <= capacity;      // capacity exceeded: flagged by the scan
            if (valid) {
                r = load_bin_rec(rec, it, n);
                nt = rec_tiles(r);
            }
        }
        if (valid && nt <= kSmallRect) {
            const ViewDev &V = vt.v[r.v];
            for (int ty = r.y0; ty <= r.y1; ++ty)
                for (int tx = r.x0; tx <= r.x1; ++tx) {
                    if (!keep_tile(vt, tmax, ellipse, r, tx, ty)) continue;
                    pkey[o] = (uint32_t)(V.tile_off + ty * V.tiles_x + tx);
                    pval[o] = it;
                    ++o;
                }
        }
        unsigned big = __ballot_sync(0xffffffffu, valid && nt > kSmallRect);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const BinRec q = shfl_rec(r, src);
            const uint32_t qit = __shfl_sync(0xffffffffu, it, src);
            long long qo = __shfl_sync(0xffffffffu, o, src);
            const ViewDev &V = vt.v[q.v];
            const int nx = q.x1 - q.x0 + 1, ntot = nx * (q.y1 - q.y0 + 1);
            for (int t0 = 0; t0 < ntot; t0 += 32) {
                const int t = t0 + lane;
                const int tx = q.x0 + t % nx, ty = q.y0 + t / nx;
                const bool kept = t < ntot && keep_tile(vt, tmax, ellipse, q, tx, ty);
                const unsigned km = __ballot_sync(0xffffffffu, kept);
                if (kept) {
                    const long long at = qo + __popc(km & lt);
                    pkey[at] = (uint32_t)(V.tile_off + ty * V.tiles_x + tx);
                    pval[at] = qit;
                }
                qo += __popc(km);
            }
        }
    }
}

// pairs to sort: all of them, or none when the capacity was exceeded (the
// emitted array then has unwritten slots; the caller re-runs with more room)
__global__ void clamp_count_kernel(const long long *total, long long capacity, long long *n_out) {
    long long t = *total;
    *n_out = t <= capacity ? t : 0;
}

// [begin, end) of each tile's run in the sorted keys
__global__ void __launch_bounds__(256)
tile_ranges_kernel(const uint32_t *__restrict__ keys, const long long *n_dev,
                   uint32_t n_tiles, uint32_t *__restrict__ ranges) {
    const long long n = *n_dev;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (k >= n_tiles) continue;
        if (i == 0 || keys[i - 1] != k) ranges[2 * (size_t)k] = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) ranges[2 * (size_t)k + 1] = (uint32_t)(i + 1);
    }
}

int tile_key_passes(int total_tiles) {
    int bits = 1;
    while ((1ll << bits) < (long long)total_tiles) ++bits;
    return (bits + 7) / 8;
}

struct BinWs {
    uint32_t *cnt, *flag, *vpos, *dkey0, *dkey1, *ditem0, *ditem1, *offs;
    uint32_t *pkey0, *pkey1, *pval_tmp;
    long long *n_vis, *n_sort;
    ScanWs scan;
    SortWs sort;
};

BinWs carve(void *ws, long long m, long long cap, size_t *bytes) {
    WsCarver c(ws);
    BinWs b;
    b.cnt = c.take<uint32_t>(m);
    b.flag = c.take<uint32_t>(m);
    b.vpos = c.take<uint32_t>(m);
    b.dkey0 = c.take<uint32_t>(m);
    b.dkey1 = c.take<uint32_t>(m);
    b.ditem0 = c.take<uint32_t>(m);
    b.ditem1 = c.take<uint32_t>(m);
    b.offs = c.take<uint32_t>(m);
    b.pkey0 = c.take<uint32_t>(cap);
    b.pkey1 = c.take<uint32_t>(cap);
    b.pval_tmp = c.take<uint32_t>(cap);
    b.n_vis = c.take<long long>(1);
    b.n_sort = c.take<long long>(1);
    b.scan.tile_status = c.take<unsigned long long>(scan_tiles(m) + 1);
    b.scan.ticket = c.take<unsigned int>(1);
    long long mt = sort_tiles(m > cap ? m : cap) + 1;
    b.sort.max_tiles = mt;
    b.sort.hist = c.take<uint32_t>(4 * 256);
    b.sort.lookback = c.take<uint32_t>((size_t)4 * 256 * mt);
    b.sort.ticket = c.take<unsigned int>(4);
    *bytes = c.off + 256;
    return b;
}

int grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 148 * 16) g = 148 * 16;
    return (int)g;
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" size_t hm_bin_sort_workspace_size(const hm_camera *cams, int32_t n_views, int32_t n,
                                             int64_t capacity, const hm_options *opt) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt) || n < 0 || capacity < 0) return 0;
    size_t bytes = 0;
    carve(nullptr, (long long)n_views * n, capacity, &bytes);
    return bytes;
}

extern "C" hm_status hm_bin_sort(const hm_camera *cams, int32_t n_views, int32_t n,
                                 const void *records, const float *tile_max_depth,
                                 const hm_options *opt, uint32_t *pair_vals, int64_t capacity,
                                 int64_t *n_pairs_out, uint32_t *tile_ranges, int32_t *d_status,
                                 void *ws, size_t ws_bytes, void *stream) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt)) return HM_ERR_INVALID_ARG;
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (capacity < 0 || capacity > HM_MAX_PAIRS) return fail(HM_ERR_INVALID_ARG, "capacity out of range");
    if ((long long)n_views * n >= (1ll << 31)) return fail(HM_ERR_INVALID_ARG, "n_views * n too large");
    if (!n_pairs_out || !tile_ranges || (n > 0 && !records) || (capacity > 0 && !pair_vals))
        return fail(HM_ERR_INVALID_ARG, "null pointer");
    if ((uintptr_t)records & 15) return fail(HM_ERR_INVALID_ARG, "records must be 16-byte aligned");
    const long long m = (long long)n_views * n;
    size_t need = 0;
    carve(nullptr, m, capacity, &need);
    if (!ws || ws_bytes < need) return fail(HM_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    BinWs b = carve(ws, m, capacity, &need);
    const Record *rec = reinterpret_cast<const Record *>(records);
    const float *tmax = opt->mesh_cull ? tile_max_depth : nullptr;
    cudaError_t e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)vt.total_tiles, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (m == 0) return cuda_status(cudaMemsetAsync(n_pairs_out, 0, sizeof(long long), s));

    // 1. kept-tile counts per record
    bin_count_kernel<<<grid_for(m, 256), 256, 0, s>>>(vt, n, rec, tmax, opt->ellipse_cull, b.cnt, b.flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    // 2. compact the visible records (count > 0) and sort them by depth
    //    (4 digit passes; the result lands back in dkey0/ditem0)
    e = launch_scan(b.flag, nullptr, b.vpos, m, b.n_vis, -1, d_status, b.scan, s);
    if (e != cudaSuccess) return cuda_status(e);
    bin_compact_kernel<<<grid_for(m, 256), 256, 0, s>>>(m, rec, b.cnt, b.vpos, b.dkey0, b.ditem0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    e = launch_radix_sort(b.dkey0, b.ditem0, b.dkey1, b.ditem1, b.n_vis, m, 4, false, d_status,
                          b.sort, s);
    if (e != cudaSuccess) return cuda_status(e);
    // 3. pair offsets in depth order; pair count and capacity check
    e = launch_scan(b.cnt, b.ditem0, b.offs, m, (long long *)n_pairs_out, capacity, d_status, b.scan, s,
                    b.n_vis);
    if (e != cudaSuccess) return cuda_status(e);
    clamp_count_kernel<<<1, 1, 0, s>>>((const long long *)n_pairs_out, capacity, b.n_sort);
    // 4. emit (tile, record) pairs; the final radix pass must land in pair_vals
    const int passes = tile_key_passes(vt.total_tiles);
    uint32_t *v0 = (passes & 1) ? b.pval_tmp : pair_vals;
    uint32_t *v1 = (passes & 1) ? pair_vals : b.pval_tmp;
    bin_emit_kernel<<<grid_for(m, 256), 256, 0, s>>>(vt, n, rec, tmax, opt->ellipse_cull, b.ditem0, b.n_vis,
                                                      b.cnt, b.offs, capacity, b.pkey0, v0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    // 5. stable sort of the pairs by tile
    e = launch_radix_sort(b.pkey0, v0, b.pkey1, v1, b.n_sort, capacity, passes, false, d_status,
                          b.sort, s);
    if (e != cudaSuccess) return cuda_status(e);
    const uint32_t *kfinal = (passes & 1) ? b.pkey1 : b.pkey0;
    // 6. tile ranges
    tile_ranges_kernel<<<grid_for(capacity, 256), 256, 0, s>>>(kfinal, b.n_sort, (uint32_t)vt.total_tiles,
                                                                 tile_ranges);
    return cuda_status(cudaGetLastError());
}
