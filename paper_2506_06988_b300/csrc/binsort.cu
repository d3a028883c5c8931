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

__device__ __forceinline__ bool tile_kept(const float *tmax, int gt, float depth) {
    return tmax == nullptr || depth < tmax[gt];
}

// d^2 along one edge of the rectangle: the edge's coordinate is fixed at e,
// the other coordinate ranges over [lo, hi]; the 1-D quadratic's minimiser
// is clamped into the range
__device__ __forceinline__ float edge_min(float p, float q, float r, float e, float lo, float hi) {
    // d^2 = p e^2 + 2 q e f + r f^2 over f in [lo, hi]
    const float f = fminf(hi, fmaxf(lo, -q * e / r));
    return fmaf(p * e, e, fmaf(2.f * q * e, f, r * f * f));
}

// Does the 3-sigma ellipse (conic a,b,c at mean m) reach the rectangle of
// the tile's in-image pixel centres?  The minimum of the convex quadratic
// d^2 over the rectangle is 0 if the mean is inside, else it lies on the
// boundary; 9 is inflated by 0.2% so the test stays a superset of the
// blend's FP32 per-pixel test.
__device__ __forceinline__ bool ellipse_hits(const ViewDev &V, int TW, int TH, int tx, int ty,
                                             float mx, float my, float a, float b, float c) {
    const float x0 = (float)(tx * TW) + 0.5f - mx;
    const float x1 = (float)(min((tx + 1) * TW, V.W) - 1) + 0.5f - mx;
    const float y0 = (float)(ty * TH) + 0.5f - my;
    const float y1 = (float)(min((ty + 1) * TH, V.H) - 1) + 0.5f - my;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
    float m = fminf(edge_min(a, b, c, x0, y0, y1), edge_min(a, b, c, x1, y0, y1));
    m = fminf(m, fminf(edge_min(c, b, a, y0, x0, x1), edge_min(c, b, a, y1, x0, x1)));
    return m <= 9.0f * 1.002f;
}

// per record: number of kept tiles, and the depth-sort key
__global__ void __launch_bounds__(256)
bin_count_kernel(ViewTable vt, int n, const Record *__restrict__ rec,
                 const float *__restrict__ tmax, int ellipse, uint32_t *__restrict__ cnt,
                 uint32_t *__restrict__ dkey) {
    const long long m = (long long)vt.n_views * n;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < m;
         it += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(it / n);
        const ViewDev &V = vt.v[v];
        const float4 a = rec[it].a;
        const float4 b = rec[it].b;
        const float4 c = rec[it].c;
        int x0, x1, y0, y1;
        unpack_range(__float_as_uint(b.w), x0, x1);
        unpack_range(__float_as_uint(c.w), y0, y1);
        uint32_t k = 0;
        if (x0 <= x1 && y0 <= y1) {
            if (tmax == nullptr && !ellipse) {
                k = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
            } else {
                for (int ty = y0; ty <= y1; ++ty) {
                    const int row = V.tile_off + ty * V.tiles_x;
                    for (int tx = x0; tx <= x1; ++tx)
                        k += tile_kept(tmax, row + tx, b.z) &&
                             (!ellipse || ellipse_hits(V, vt.tile_w, vt.tile_h, tx, ty, a.x, a.y, a.z, a.w, b.x));
                }
            }
        }
        cnt[it] = k;
        dkey[it] = k ? __float_as_uint(b.z) : 0xFFFFFFFFu;
    }
}

// per depth-sorted record: write its (tile, record) pairs at its scan offset
__global__ void __launch_bounds__(256)
bin_emit_kernel(ViewTable vt, int n, const Record *__restrict__ rec,
                const float *__restrict__ tmax, int ellipse, const uint32_t *__restrict__ sorted_items,
                const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ offs,
                long long capacity, uint32_t *__restrict__ pkey, uint32_t *__restrict__ pval) {
    const long long m = (long long)vt.n_views * n;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const uint32_t it = sorted_items[j];
        const uint32_t k = cnt[it];
        if (k == 0) continue;
        long long o = offs[j];
        if (o + k > capacity) continue;          // capacity exceeded: flagged by the scan
        const int v = (int)(it / (uint32_t)n);
        const ViewDev &V = vt.v[v];
        const float4 a = rec[it].a;
        const float4 b = rec[it].b;
        const float4 c = rec[it].c;
        int x0, x1, y0, y1;
        unpack_range(__float_as_uint(b.w), x0, x1);
        unpack_range(__float_as_uint(c.w), y0, y1);
        for (int ty = y0; ty <= y1; ++ty) {
            const int row = V.tile_off + ty * V.tiles_x;
            for (int tx = x0; tx <= x1; ++tx) {
                if (!tile_kept(tmax, row + tx, b.z)) continue;
                if (ellipse && !ellipse_hits(V, vt.tile_w, vt.tile_h, tx, ty, a.x, a.y, a.z, a.w, b.x)) continue;
                pkey[o] = (uint32_t)(row + tx);
                pval[o] = it;
                ++o;
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
    uint32_t *cnt, *dkey0, *dkey1, *ditem0, *ditem1, *offs;
    uint32_t *pkey0, *pkey1, *pval_tmp;
    long long *n_items, *n_sort;
    ScanWs scan;
    SortWs sort;
};

BinWs carve(void *ws, long long m, long long cap, size_t *bytes) {
    WsCarver c(ws);
    BinWs b;
    b.cnt = c.take<uint32_t>(m);
    b.dkey0 = c.take<uint32_t>(m);
    b.dkey1 = c.take<uint32_t>(m);
    b.ditem0 = c.take<uint32_t>(m);
    b.ditem1 = c.take<uint32_t>(m);
    b.offs = c.take<uint32_t>(m);
    b.pkey0 = c.take<uint32_t>(cap);
    b.pkey1 = c.take<uint32_t>(cap);
    b.pval_tmp = c.take<uint32_t>(cap);
    b.n_items = c.take<long long>(1);
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

    // 1. counts and depth keys
    bin_count_kernel<<<grid_for(m, 256), 256, 0, s>>>(vt, n, rec, tmax, opt->ellipse_cull, b.cnt, b.dkey0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    // 2. depth sort of the records (4 digit passes; result back in dkey0/ditem0)
    if ((e = launch_fill_i64(b.n_items, m, s)) != cudaSuccess) return cuda_status(e);
    e = launch_radix_sort(b.dkey0, b.ditem0, b.dkey1, b.ditem1, b.n_items, m, 4, true, d_status,
                          b.sort, s);
    if (e != cudaSuccess) return cuda_status(e);
    // 3. pair offsets in depth order; pair count and capacity check
    e = launch_scan(b.cnt, b.ditem0, b.offs, m, (long long *)n_pairs_out, capacity, d_status, b.scan, s);
    if (e != cudaSuccess) return cuda_status(e);
    clamp_count_kernel<<<1, 1, 0, s>>>((const long long *)n_pairs_out, capacity, b.n_sort);
    // 4. emit (tile, record) pairs; the final radix pass must land in pair_vals
    const int passes = tile_key_passes(vt.total_tiles);
    uint32_t *v0 = (passes & 1) ? b.pval_tmp : pair_vals;
    uint32_t *v1 = (passes & 1) ? pair_vals : b.pval_tmp;
    bin_emit_kernel<<<grid_for(m, 256), 256, 0, s>>>(vt, n, rec, tmax, opt->ellipse_cull, b.ditem0, b.cnt, b.offs,
                                                      capacity, b.pkey0, v0);
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
