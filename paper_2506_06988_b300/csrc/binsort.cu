// binsort.cu -- tile binning and the per-tile depth sort of (Gaussian, tile)
// pairs (the "tile-wise sorting" of the splatting rasteriser, Sec. 1).
//
// Each tile's list must be ordered by (FP32 depth, Gaussian index).  The
// pairs are bucketed by tile first and each tile's bucket is then sorted on
// its own (a segmented sort), instead of a global radix sort on a
// (tile, depth) key:
//  1. count: per (record, tile) of each record's tile rectangle, whether the
//     tile is kept (mesh cull, ellipse test), and per tile the number of
//     records that keep it (atomic counts); the candidates of a block of
//     records are spread evenly over the CTA's threads (load-balanced
//     expansion: most records are culled, and the visible ones span from
//     one to a thousand tiles);
//  2. scan of the per-tile counts: each tile's [begin, end) in the output,
//     the pair count and the capacity check;
//  3. emit: the same expansion; every kept (record, tile) writes the 64-bit
//     key (depth bits << 32 | record index) into its tile's bucket at an
//     atomically taken slot (bucket order is arbitrary at this point);
//  4. sort each bucket by that key -- a warp per tile in registers (bitonic)
//     for up to 256 pairs, a CTA in shared memory (radix) for up to 4096, a
//     CTA with radix passes through global memory beyond -- and write the
//     record indices.
// Positive FP32 depths order like their bit patterns, and all records of a
// tile belong to one camera, so the key order is (depth, Gaussian index).
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
    float mx, my, a, b, c, depth;   // mean, conic, depth key
    int x0, x1, y0, y1, v;          // tile rectangle, camera
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
    r.depth = B.z;
    unpack_range(__float_as_uint(B.w), r.x0, r.x1);
    unpack_range(__float_as_uint(C.w), r.y0, r.y1);
    r.v = (int)((uint32_t)it / (uint32_t)n);   // record indices stay below 2^31
    return r;
}

__device__ __forceinline__ int rec_tiles(const BinRec &r) {
    return (r.x0 <= r.x1 && r.y0 <= r.y1) ? (r.x1 - r.x0 + 1) * (r.y1 - r.y0 + 1) : 0;
}

// Is the pair (record, tile) kept (ra, rc = 1 / conic_xx, 1 / conic_yy)?  Mesh cull: the tile's farthest mesh depth
// must lie behind the record (Sec. 3.4 blends only D_gs < D_m).  Ellipse
// test: the 3-sigma ellipse must reach the rectangle of the tile's in-image
// pixel centres -- the minimum of the convex d^2 over the rectangle is 0 with
// the mean inside, else on an edge; 9 is inflated by 0.2% so the test stays
// a superset of the blend's FP32 per-pixel test.
__device__ __forceinline__ bool keep_tile(const ViewTable &vt, const float *tmax, int ellipse,
                                          const BinRec &r, float ra, float rc, int tx, int ty) {
    const ViewDev &V = vt.v[r.v];
    if (tmax != nullptr && !(r.depth < tmax[V.tile_off + ty * V.tiles_x + tx])) return false;
    if (!ellipse) return true;
    const float x0 = (float)(tx * vt.tile_w) + 0.5f - r.mx;
    const float x1 = (float)(min((tx + 1) * vt.tile_w, V.W) - 1) + 0.5f - r.mx;
    const float y0 = (float)(ty * vt.tile_h) + 0.5f - r.my;
    const float y1 = (float)(min((ty + 1) * vt.tile_h, V.H) - 1) + 0.5f - r.my;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
    float m = fminf(edge_min(r.a, r.b, r.c, rc, x0, y0, y1), edge_min(r.a, r.b, r.c, rc, x1, y0, y1));
    m = fminf(m, fminf(edge_min(r.c, r.b, r.a, ra, y0, x0, x1), edge_min(r.c, r.b, r.a, ra, y1, x0, x1)));
    return m <= 9.0f * 1.002f;
}

// Binning of a block of records by load-balanced expansion.  A CTA takes
// kBinThreads records; each thread loads one and counts the tiles of its
// rectangle (0 for a culled record), a block-wide exclusive scan lays the
// records' (record, tile) candidates end to end, and every thread of the
// CTA then takes candidates c = t, t + kBinThreads, ... : the record is the
// last slot whose offset is <= c (binary search over the offsets in shared
// memory), the tile follows from c - offset.  A record spanning a thousand
// tiles and a block of single-tile records keep every thread equally busy,
// and a CTA's candidate loads and atomics are in flight together.  Each
// candidate takes the mesh cull and the ellipse test (keep_tile); count and
// emission run the same expansion, so they keep the same pairs.  The count
// walks all records in index order and appends the ones with a non-empty
// rectangle (a few percent at 1080p) to a list; the emission walks only
// that list.
constexpr int kBinThreads = 256;
constexpr int kEmitRecs = 64;      // listed records per block of the emission

struct BinBlock {
    uint32_t off[kBinThreads + 1];   // exclusive prefix of the rectangles' tile counts; [256] = total
    uint32_t wsum[kBinThreads / 32];
    float mx[kBinThreads], my[kBinThreads], a[kBinThreads], b[kBinThreads], c[kBinThreads];
    float ra[kBinThreads], rc[kBinThreads], depth[kBinThreads];
    int x0[kBinThreads], y0[kBinThreads], nx[kBinThreads], v[kBinThreads];
    uint32_t idx[kBinThreads];       // record index
};

// Loads the block's records -- for t < nrec and first + t < limit, record
// `first + t` (list == nullptr) or list[first + t] -- and scans their
// rectangle sizes; returns the total, `cnt` the thread's own record's count.
__device__ __forceinline__ uint32_t bin_block_load(BinBlock &S, const Record *__restrict__ rec,
                                                   const uint32_t *__restrict__ list, uint32_t first,
                                                   uint32_t limit, int nrec, int n, uint32_t &cnt,
                                                   uint32_t &it) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    cnt = 0;
    it = 0;
    if (t < nrec && first + (uint32_t)t < limit) {
        it = list ? list[first + t] : first + (uint32_t)t;
        const BinRec r = load_bin_rec(rec, it, n);
        cnt = (uint32_t)rec_tiles(r);
        if (cnt) {
            S.mx[t] = r.mx; S.my[t] = r.my;
            S.a[t] = r.a; S.b[t] = r.b; S.c[t] = r.c;
            S.ra[t] = 1.f / r.a; S.rc[t] = 1.f / r.c;
            S.depth[t] = r.depth;
            S.x0[t] = r.x0; S.y0[t] = r.y0; S.nx[t] = r.x1 - r.x0 + 1; S.v[t] = r.v;
            S.idx[t] = it;
        }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) S.wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t ws = lane < kBinThreads / 32 ? S.wsum[lane] : 0u;
        uint32_t wi = ws;
#pragma unroll
        for (int o = 1; o < kBinThreads / 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kBinThreads / 32) S.wsum[lane] = wi - ws;          // exclusive over warps
        if (lane == kBinThreads / 32 - 1) S.off[kBinThreads] = wi;   // total
    }
    __syncthreads();
    S.off[t] = S.wsum[w] + incl - cnt;
    __syncthreads();
    return S.off[kBinThreads];
}

// Candidate c of the block: its record slot j and tile (tx, ty); true if
// the pair is kept.
__device__ __forceinline__ bool bin_candidate(const BinBlock &S, const ViewTable &vt, const float *tmax,
                                              int ellipse, uint32_t c, int &j, int &tx, int &ty) {
    int lo = 0, hi = kBinThreads;                    // off[lo] <= c < off[hi]
#pragma unroll
    for (int step = 0; step < 8; ++step) {
        const int mid = (lo + hi) >> 1;
        if (S.off[mid] <= c) lo = mid;
        else hi = mid;
    }
    j = lo;
    const uint32_t o = c - S.off[j];
    const int nx = S.nx[j];
    tx = S.x0[j] + (int)(o % (uint32_t)nx);
    ty = S.y0[j] + (int)(o / (uint32_t)nx);
    BinRec r;
    r.mx = S.mx[j]; r.my = S.my[j]; r.a = S.a[j]; r.b = S.b[j]; r.c = S.c[j]; r.depth = S.depth[j];
    r.v = S.v[j];
    return keep_tile(vt, tmax, ellipse, r, S.ra[j], S.rc[j], tx, ty);
}

// Per tile: the number of records that keep it (atomic counts); the
// records with a non-empty rectangle are appended to `vis` (order
// arbitrary: the emitted keys carry the record index).
__global__ void __launch_bounds__(kBinThreads)
bin_count_kernel(ViewTable vt, int n, const Record *__restrict__ rec, const float *__restrict__ tmax,
                 int ellipse, uint32_t *__restrict__ tile_cnt, uint32_t *__restrict__ vis,
                 unsigned int *__restrict__ n_vis) {
    __shared__ BinBlock S;
    uint32_t mine, it;
    const uint32_t total = bin_block_load(S, rec, nullptr, blockIdx.x * kBinThreads,
                                          (uint32_t)((long long)vt.n_views * n), kBinThreads, n, mine, it);
    {
        const int lane = threadIdx.x & 31;
        const unsigned bal = __ballot_sync(0xffffffffu, mine > 0);
        unsigned base = 0;
        if (lane == 0 && bal) base = atomicAdd(n_vis, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (mine > 0) vis[base + __popc(bal & ((1u << lane) - 1u))] = it;
    }
    for (uint32_t c = threadIdx.x; c < total; c += kBinThreads) {
        int j, tx, ty;
        if (bin_candidate(S, vt, tmax, ellipse, c, j, tx, ty)) {
            const ViewDev &V = vt.v[S.v[j]];
            // a reduction (no return value): hot tiles' adds queue in L2
            if (hm_check(tx >= 0 && tx < V.tiles_x && ty >= 0 && ty < V.tiles_y))
                atomicAdd(&tile_cnt[V.tile_off + ty * V.tiles_x + tx], 1u);
        }
    }
}

// pairs to sort: all of them, or none when the capacity was exceeded
__global__ void clamp_count_kernel(const long long *total, long long capacity, long long *n_out) {
    long long t = *total;
    *n_out = t <= capacity ? t : 0;
}

// Every kept (record, tile): the 64-bit key (depth bits << 32 | record
// index) into the tile's bucket, at a slot taken from the tile's cursor
// (initialised to the bucket's start); nothing is written when the
// capacity was exceeded.  The CTAs walk the list of records with a
// non-empty rectangle, kEmitRecs at a time (grid-stride): such a record
// spans tens of tiles, so a few records already give every thread of the
// CTA candidates, and many CTAs keep the cursors' returning atomics in
// flight together.
__global__ void __launch_bounds__(kBinThreads)
bin_emit_kernel(ViewTable vt, int n, const Record *__restrict__ rec, const float *__restrict__ tmax,
                int ellipse, const uint32_t *__restrict__ vis, const unsigned int *n_vis,
                uint32_t *__restrict__ cursor, const long long *n_sort, unsigned long long *__restrict__ keys) {
    if (*n_sort == 0) return;
    __shared__ BinBlock S;
    const uint32_t nv = *n_vis;
    for (uint32_t first = blockIdx.x * kEmitRecs; first < nv; first += gridDim.x * kEmitRecs) {
        __syncthreads();                             // the previous block's shared reads are done
        uint32_t mine, it;
        const uint32_t total = bin_block_load(S, rec, vis, first, nv, kEmitRecs, n, mine, it);
        for (uint32_t c = threadIdx.x; c < total; c += kBinThreads) {
            int j, tx, ty;
            if (bin_candidate(S, vt, tmax, ellipse, c, j, tx, ty)) {
                const ViewDev &V = vt.v[S.v[j]];
                if (!hm_check(tx >= 0 && tx < V.tiles_x && ty >= 0 && ty < V.tiles_y)) continue;
                const uint32_t slot = atomicAdd(&cursor[V.tile_off + ty * V.tiles_x + tx], 1u);
                if (hm_check(slot < (unsigned long long)*n_sort))
                    keys[slot] = ((unsigned long long)__float_as_uint(S.depth[j]) << 32) | S.idx[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// segmented sort of the tile buckets
// ---------------------------------------------------------------------------

// The lanes of the warp whose 9-bit value d (a digit, or 256 for no key)
// equals this lane's: one ballot per bit, keeping the lanes that agree on it.
__device__ __forceinline__ uint32_t same_digit_lanes(uint32_t d) {
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const uint32_t one = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        m &= ((d >> b) & 1u) ? one : ~one;
    }
    return m;
}
constexpr int kWarpSeg = 256;      // bucket sizes sorted by one warp in registers
constexpr int kMidSeg = 1024;      // ... by a 128-thread CTA in shared memory (radix)
constexpr int kSegMax = 4096;      // ... by a 256-thread CTA in shared memory (radix)
constexpr int kBigSeg = 8192;      // ... by a 512-thread CTA in shared memory (radix)

// compare-exchange of a (low, high) element pair for an ascending (asc) or
// descending bitonic stage: afterwards lo holds the min if asc, else the max
__device__ __forceinline__ void cmp_swap(unsigned long long &lo, unsigned long long &hi, bool asc) {
    const bool sw = (lo > hi) == asc;
    const unsigned long long a = lo, b = hi;
    lo = sw ? b : a;
    hi = sw ? a : b;
}

// in-lane compare-exchange stage of warp_bitonic: slots sl and sl ^ JS of
// each lane (partner distance 32 JS elements)
template <int E, int JS>
__device__ __forceinline__ void lane_stage(unsigned long long (&v)[E], int lane, int k) {
#pragma unroll
    for (int sl = 0; sl < E; ++sl)
        if (!(sl & JS)) cmp_swap(v[sl], v[sl | JS], ((lane + 32 * sl) & k) == 0);
}

// Bitonic sort of the 32 E keys of a warp held in registers: element
// e = lane + 32 s sits in lane e % 32, slot s.  Stages whose partner
// distance j is >= 32 pair two slots of the same lane; shorter ones pair the
// same slot of lanes lane and lane ^ j (one shuffle per slot).  The stage
// loops run at run time (only the slot loop is unrolled), which keeps the
// code small enough for the instruction cache.
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&v)[E], int lane) {
    constexpr int N = 32 * E;
#pragma unroll 1
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll 1
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int js = j >> 5;
                if (E > 1 && js == 1) lane_stage<E, 1>(v, lane, k);
                if (E > 2 && js == 2) lane_stage<E, (E > 2 ? 2 : 1)>(v, lane, k);
                if (E > 4 && js == 4) lane_stage<E, (E > 4 ? 4 : 1)>(v, lane, k);
                if (E > 8 && js == 8) lane_stage<E, (E > 8 ? 8 : 1)>(v, lane, k);
                if (E > 16 && js == 16) lane_stage<E, (E > 16 ? 16 : 1)>(v, lane, k);
            } else {
                const bool low = (lane & j) == 0;
#pragma unroll
                for (int sl = 0; sl < E; ++sl) {
                    const unsigned long long p = __shfl_xor_sync(0xffffffffu, v[sl], j);
                    // the lower element keeps the min in an ascending block
                    const bool take_min = low == (((lane + 32 * sl) & k) == 0);
                    v[sl] = take_min ? (p < v[sl] ? p : v[sl]) : (p > v[sl] ? p : v[sl]);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void warp_sort_bucket(const unsigned long long *__restrict__ keys,
                                                 uint32_t *__restrict__ vals, uint32_t off, uint32_t cnt,
                                                 int lane) {
    unsigned long long v[E];
#pragma unroll
    for (int sl = 0; sl < E; ++sl) {
        const uint32_t e = lane + 32 * sl;
        v[sl] = e < cnt ? keys[off + e] : ~0ull;
    }
    warp_bitonic<E>(v, lane);
#pragma unroll
    for (int sl = 0; sl < E; ++sl) {
        const uint32_t e = lane + 32 * sl;
        if (e < cnt) vals[off + e] = (uint32_t)v[sl];
    }
}

// Warp per tile (grid-stride): writes the tile's range; buckets of up to 256
// keys are sorted in registers (the smallest power-of-two slot count that
// holds them); larger buckets go to the mid-size (up to 4096 keys, radix
// sorted by a CTA) or the large list.  Nothing when the capacity was
// exceeded (ranges stay empty).
__global__ void __launch_bounds__(256)
seg_sort_small_kernel(uint32_t n_tiles, const uint32_t *__restrict__ tile_off,
                      const uint32_t *__restrict__ tile_cnt, const long long *n_sort,
                      const unsigned long long *__restrict__ keys, uint32_t *__restrict__ vals,
                      uint32_t *__restrict__ ranges, uint32_t *__restrict__ mid_list,
                      unsigned int *__restrict__ mid_count, uint32_t *__restrict__ big_list,
                      unsigned int *__restrict__ big_count) {
    if (*n_sort == 0) return;
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t gt = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gt < n_tiles; gt += nw) {
        uint32_t off = tile_off[gt], cnt = tile_cnt[gt];
        // (checked build: a bucket beyond the pairs is left empty)
        if (!hm_check((unsigned long long)off + cnt <= (unsigned long long)*n_sort)) off = cnt = 0;
        if (lane == 0) {
            ranges[2 * (size_t)gt] = off;
            ranges[2 * (size_t)gt + 1] = off + cnt;
        }
        if (cnt == 0) continue;
        if (cnt == 1) {
            if (lane == 0) vals[off] = (uint32_t)keys[off];
        } else if (cnt <= 32) {
            warp_sort_bucket<1>(keys, vals, off, cnt, lane);
        } else if (cnt <= 64) {
            warp_sort_bucket<2>(keys, vals, off, cnt, lane);
        } else if (cnt <= 128) {
            warp_sort_bucket<4>(keys, vals, off, cnt, lane);
        } else if (cnt <= (uint32_t)kWarpSeg) {
            warp_sort_bucket<8>(keys, vals, off, cnt, lane);
        } else if (lane == 0) {
            if (cnt <= (uint32_t)kMidSeg) mid_list[atomicAdd(mid_count, 1u)] = gt;
            else big_list[atomicAdd(big_count, 1u)] = gt;
        }
    }
}

// ---- CTA radix sort of one bucket of up to CAP keys in shared memory.
// The sort key is the depth (the high word of the 64-bit pair key) with the
// record index as payload: 4 stable LSD passes of 8 bits, skipping passes in
// which every key has the same digit.  A pass ranks the keys warp by warp
// (one ballot per digit bit gives each key its rank among equal digits in
// input order),
// turns the per-warp digit counts into offsets and scatters -- stable, so
// equal depths keep their input order, which the emission left arbitrary:
// a final fix-up sorts each run of equal depths by record index, which
// makes the result the (depth, index) order.
template <int THREADS, int CAP>
struct RadixSmem {
    static constexpr int kWarps = THREADS / 32;
    uint32_t k[2][CAP];
    uint32_t v[2][CAP];
    uint32_t whist[kWarps][257];   // per-warp digit counts, then offsets
    uint32_t dstart[256];          // bucket-local start of each digit
    uint32_t wsum[kWarps];
    uint32_t kand, kor;
};

template <int THREADS, int CAP>
__device__ void radix_pass(RadixSmem<THREADS, CAP> &S, int src, int n, int shift) {
    constexpr int kWarps = THREADS / 32, kItems = CAP / THREADS;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = lanemask_lt();
    for (int i = t; i < kWarps * 257; i += THREADS) (&S.whist[0][0])[i] = 0;
    __syncthreads();
    // warp w ranks the contiguous chunk [w C, (w + 1) C), items in input order
    const int per = (n + THREADS - 1) / THREADS;     // items per lane
    const int C = 32 * per;
    uint32_t key[kItems], val[kItems], rank[kItems];
    int dig[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        if (j >= per) break;
        const int e = w * C + j * 32 + lane;
        const bool valid = e < n;
        key[j] = valid ? S.k[src][e] : 0u;
        val[j] = valid ? S.v[src][e] : 0u;
        const int d = valid ? (int)((key[j] >> shift) & 255u) : 256;
        dig[j] = d;
        const uint32_t peers = same_digit_lanes((uint32_t)d);
        const uint32_t before = S.whist[w][d];
        __syncwarp();
        if ((peers & lt) == 0) S.whist[w][d] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt);
    }
    __syncthreads();
    // digit d (threads take digits t, t + THREADS, ...): offsets of the warps
    // within the digit and the digit total; then an exclusive scan over the
    // 256 digits
    for (int d = t; d < 256; d += THREADS) {
        uint32_t cnt = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t c = S.whist[ww][d];
            S.whist[ww][d] = cnt;
            cnt += c;
        }
        S.dstart[d] = cnt;
    }
    __syncthreads();
    if (w == 0) {
        // 256 totals, 8 per lane: serial within the lane, shuffle scan across
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = S.dstart[lane * 8 + q];
            sum += c[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            S.dstart[lane * 8 + q] = run;
            run += c[q];
        }
    }
    __syncthreads();
    const int dst = src ^ 1;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        if (j >= per) break;
        const int d = dig[j];
        if (d < 256) {
            const uint32_t pos = S.dstart[d] + S.whist[w][d] + rank[j];
            S.k[dst][pos] = key[j];
            S.v[dst][pos] = val[j];
        }
    }
    __syncthreads();
}

// CTA per bucket of at most CAP keys (grid-stride over its list).
template <int THREADS, int CAP, int LOWER = 0>
__global__ void __launch_bounds__(THREADS)
seg_sort_radix_kernel(const uint32_t *__restrict__ list, const unsigned int *list_count,
                      const uint32_t *__restrict__ tile_off, const uint32_t *__restrict__ tile_cnt,
                      const unsigned long long *__restrict__ keys, uint32_t *__restrict__ vals) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RadixSmem<THREADS, CAP> &S = *reinterpret_cast<RadixSmem<THREADS, CAP> *>(smem_raw);
    const int t = threadIdx.x;
    const unsigned int nl = *list_count;
    for (unsigned int li = blockIdx.x; li < nl; li += gridDim.x) {
        const uint32_t gt = list[li];
        const uint32_t off = tile_off[gt];
        const int n = (int)tile_cnt[gt];
        if (n > CAP || n <= LOWER) continue;         // another tier's bucket
        if (t == 0) {
            S.kand = 0xFFFFFFFFu;
            S.kor = 0u;
        }
        __syncthreads();
        uint32_t ka = 0xFFFFFFFFu, ko = 0u;
        for (int i = t; i < n; i += THREADS) {
            const unsigned long long kv = keys[off + i];
            const uint32_t k = (uint32_t)(kv >> 32);
            S.k[0][i] = k;
            S.v[0][i] = (uint32_t)kv;
            ka &= k;
            ko |= k;
        }
        atomicAnd(&S.kand, ka);
        atomicOr(&S.kor, ko);
        __syncthreads();
        const uint32_t differ = S.kand ^ S.kor;     // bits that are not the same in every key
        int src = 0;
        for (int pass = 0; pass < 4; ++pass) {
            if (((differ >> (8 * pass)) & 255u) == 0) continue;   // one digit value: identity pass
            radix_pass<THREADS, CAP>(S, src, n, 8 * pass);
            src ^= 1;
        }
        // runs of equal depth: order by record index (a thread per run start)
        for (int i = t; i < n; i += THREADS) {
            const uint32_t k = S.k[src][i];
            if (i > 0 && S.k[src][i - 1] == k) continue;          // not a run start
            int e = i + 1;
            while (e < n && S.k[src][e] == k) ++e;
            for (int a = i + 1; a < e; ++a) {                     // insertion sort of the run
                const uint32_t x = S.v[src][a];
                int b = a - 1;
                while (b >= i && S.v[src][b] > x) {
                    S.v[src][b + 1] = S.v[src][b];
                    --b;
                }
                S.v[src][b + 1] = x;
            }
        }
        __syncthreads();
        for (int i = t; i < n; i += THREADS) vals[off + i] = S.v[src][i];
        __syncthreads();
    }
}

template <int THREADS, int CAP, int LOWER = 0>
cudaError_t launch_radix_buckets(const uint32_t *list, const unsigned int *count, const uint32_t *tile_off,
                                 const uint32_t *tile_cnt, const unsigned long long *keys, uint32_t *vals,
                                 int grid, cudaStream_t s) {
    static bool attr = false;
    const int smem = (int)sizeof(RadixSmem<THREADS, CAP>);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(seg_sort_radix_kernel<THREADS, CAP, LOWER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    seg_sort_radix_kernel<THREADS, CAP, LOWER><<<grid, THREADS, smem, s>>>(list, count, tile_off, tile_cnt, keys,
                                                                        vals);
    return cudaGetLastError();
}

// ---- buckets above kBigSeg keys: one CTA, LSD radix passes through global
// memory in chunks of kSegMax.  The depth keys are split from the record
// indices into two uint32 arrays (ping-pong between the bucket's range of
// `scratch` and of the key array itself).  One read counts every pass's
// digits; a pass then walks the chunks in order, ranks each chunk in shared
// memory exactly as radix_pass does (stable), and scatters it to
// digit start + count of the digit in earlier chunks + rank, which keeps the
// pass stable across chunks.  Runs of equal depth are then ordered by
// record index as in the in-shared-memory sort.
template <int THREADS, int CAP>
struct HugeSmem {
    RadixSmem<THREADS, CAP> r;
    uint32_t hist[4][256];
    uint32_t base[256];
    uint32_t run[256];
};

template <int THREADS, int CAP>
__device__ void huge_chunk_pass(HugeSmem<THREADS, CAP> &H, const uint32_t *ks, const uint32_t *vs,
                                uint32_t *kd, uint32_t *vd, int n0, int n, int shift) {
    constexpr int kWarps = THREADS / 32, kItems = CAP / THREADS;
    RadixSmem<THREADS, CAP> &S = H.r;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = lanemask_lt();
    for (int i = t; i < n; i += THREADS) {
        S.k[0][i] = ks[n0 + i];
        S.v[0][i] = vs[n0 + i];
    }
    for (int i = t; i < kWarps * 257; i += THREADS) (&S.whist[0][0])[i] = 0;
    __syncthreads();
    const int per = (n + THREADS - 1) / THREADS;
    const int C = 32 * per;
    uint32_t key[kItems], val[kItems], rank[kItems];
    int dig[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        if (j >= per) break;
        const int e = w * C + j * 32 + lane;
        const bool valid = e < n;
        key[j] = valid ? S.k[0][e] : 0u;
        val[j] = valid ? S.v[0][e] : 0u;
        const int d = valid ? (int)((key[j] >> shift) & 255u) : 256;
        dig[j] = d;
        const uint32_t peers = same_digit_lanes((uint32_t)d);
        const uint32_t before = S.whist[w][d];
        __syncwarp();
        if ((peers & lt) == 0) S.whist[w][d] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: the warps' offsets within the chunk's digit, chunk total
    for (int d = t; d < 256; d += THREADS) {
        uint32_t cnt = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t c = S.whist[ww][d];
            S.whist[ww][d] = cnt;
            cnt += c;
        }
        S.dstart[d] = cnt;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        if (j >= per) break;
        const int d = dig[j];
        if (d < 256) {
            const uint32_t pos = H.base[d] + H.run[d] + S.whist[w][d] + rank[j];
            kd[pos] = key[j];
            vd[pos] = val[j];
        }
    }
    __syncthreads();
    for (int d = t; d < 256; d += THREADS) H.run[d] += S.dstart[d];
    __syncthreads();
}

template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS)
seg_sort_huge_kernel(const uint32_t *__restrict__ list, const unsigned int *list_count,
                     const uint32_t *__restrict__ tile_off, const uint32_t *__restrict__ tile_cnt,
                     unsigned long long *__restrict__ keys, unsigned long long *__restrict__ scratch,
                     uint32_t *__restrict__ vals, int min_n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HugeSmem<THREADS, CAP> &H = *reinterpret_cast<HugeSmem<THREADS, CAP> *>(smem_raw);
    const int t = threadIdx.x;
    const unsigned int nl = *list_count;
    for (unsigned int li = blockIdx.x; li < nl; li += gridDim.x) {
        const uint32_t gt = list[li];
        const long long off = tile_off[gt];
        const int n = (int)tile_cnt[gt];
        if (n <= min_n) continue;                    // sorted in shared memory by a radix CTA
        // A = (depth keys, record indices) split into the scratch range,
        // B = the same layout over the key range
        uint32_t *kA = reinterpret_cast<uint32_t *>(scratch + off), *vA = kA + n;
        uint32_t *kB = reinterpret_cast<uint32_t *>(keys + off), *vB = kB + n;
        for (int i = t; i < 4 * 256; i += THREADS) (&H.hist[0][0])[i] = 0;
        if (t == 0) {
            H.r.kand = 0xFFFFFFFFu;
            H.r.kor = 0u;
        }
        __syncthreads();
        uint32_t ka = 0xFFFFFFFFu, ko = 0u;
        const int lane = t & 31;
        for (int i0 = 0; i0 < n; i0 += THREADS) {
            const int i = i0 + t;
            const bool valid = i < n;
            uint32_t k = 0;
            if (valid) {
                const unsigned long long kv = keys[off + i];
                k = (uint32_t)(kv >> 32);
                kA[i] = k;
                vA[i] = (uint32_t)kv;
                ka &= k;
                ko |= k;
            }
            // digit counts: one shared atomic per distinct digit of the warp
            // (depth digits are skewed: many keys share the high bytes)
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const uint32_t d = valid ? (k >> (8 * p)) & 255u : 256u;
                const unsigned peers = same_digit_lanes(d);
                if (valid && lane == __ffs(peers) - 1) atomicAdd(&H.hist[p][d], (unsigned)__popc(peers));
            }
        }
        atomicAnd(&H.r.kand, ka);
        atomicOr(&H.r.kor, ko);
        __syncthreads();
        const uint32_t differ = H.r.kand ^ H.r.kor;
        bool inA = true;
        for (int pass = 0; pass < 4; ++pass) {
            if (((differ >> (8 * pass)) & 255u) == 0) continue;   // one digit value: identity pass
            // digit starts of this pass (exclusive scan of the bucket's histogram)
            if (t < 32) {
                uint32_t c[8], sum = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    c[q] = H.hist[pass][t * 8 + q];
                    sum += c[q];
                }
                uint32_t incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (t >= o) incl += y;
                }
                uint32_t runv = incl - sum;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    H.base[t * 8 + q] = runv;
                    H.run[t * 8 + q] = 0;
                    runv += c[q];
                }
            }
            __syncthreads();
            const uint32_t *ks = inA ? kA : kB, *vs = inA ? vA : vB;
            uint32_t *kd = inA ? kB : kA, *vd = inA ? vB : vA;
            for (int c0 = 0; c0 < n; c0 += CAP)
                huge_chunk_pass<THREADS, CAP>(H, ks, vs, kd, vd, c0, min(CAP, n - c0), 8 * pass);
            inA = !inA;
        }
        __syncthreads();
        uint32_t *kf = inA ? kA : kB, *vf = inA ? vA : vB;
        // runs of equal depth: order by record index (a thread per run start)
        for (int i = t; i < n; i += THREADS) {
            const uint32_t k = kf[i];
            if (i > 0 && kf[i - 1] == k) continue;
            int e = i + 1;
            while (e < n && kf[e] == k) ++e;
            for (int a = i + 1; a < e; ++a) {
                const uint32_t x = vf[a];
                int b = a - 1;
                while (b >= i && vf[b] > x) {
                    vf[b + 1] = vf[b];
                    --b;
                }
                vf[b + 1] = x;
            }
        }
        __syncthreads();
        for (int i = t; i < n; i += THREADS) vals[off + i] = vf[i];
        __syncthreads();
    }
}

struct BinWs {
    uint32_t *tile_cnt, *tile_off, *tile_fill, *mid_list, *big_list, *vis;
    unsigned long long *keys, *scratch;
    unsigned int *counts;   // [0] mid-size buckets (<= kMidSeg), [1] larger buckets, [2] listed records
    long long *n_sort;
    ScanWs scan;
};

BinWs carve(void *ws, long long m, long long cap, long long tiles, size_t *bytes) {
    WsCarver c(ws);
    BinWs b;
    b.tile_cnt = c.take<uint32_t>(tiles);
    b.tile_off = c.take<uint32_t>(tiles);
    b.tile_fill = c.take<uint32_t>(tiles);
    b.mid_list = c.take<uint32_t>(tiles);
    b.big_list = c.take<uint32_t>(tiles);
    b.keys = c.take<unsigned long long>(cap);
    b.scratch = c.take<unsigned long long>(cap);
    b.vis = c.take<uint32_t>(m);
    b.counts = c.take<unsigned int>(3);
    b.n_sort = c.take<long long>(1);
    b.scan.tile_status = c.take<unsigned long long>(scan_tiles(tiles) + 1);
    b.scan.ticket = c.take<unsigned int>(1);
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
    carve(nullptr, (long long)n_views * n, capacity, vt.total_tiles, &bytes);
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
    const long long T = vt.total_tiles;
    size_t need = 0;
    carve(nullptr, m, capacity, T, &need);
    if (!ws || ws_bytes < need) return fail(HM_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    BinWs b = carve(ws, m, capacity, T, &need);
    const Record *rec = reinterpret_cast<const Record *>(records);
    const float *tmax = opt->mesh_cull ? tile_max_depth : nullptr;
    cudaError_t e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)T, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (m == 0) return cuda_status(cudaMemsetAsync(n_pairs_out, 0, sizeof(long long), s));
    if ((e = cudaMemsetAsync(b.tile_cnt, 0, sizeof(uint32_t) * (size_t)T, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(b.counts, 0, 3 * sizeof(unsigned int), s)) != cudaSuccess)
        return cuda_status(e);

    // 1. kept tiles per record, records per tile
    const unsigned rgrid = (unsigned)((m + kBinThreads - 1) / kBinThreads);
    bin_count_kernel<<<rgrid, kBinThreads, 0, s>>>(vt, n, rec, tmax, opt->ellipse_cull, b.tile_cnt, b.vis,
                                                   b.counts + 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    // 2. tile offsets, pair count and capacity check
    e = launch_scan(b.tile_cnt, nullptr, b.tile_off, T, (long long *)n_pairs_out, capacity, d_status, b.scan, s);
    if (e != cudaSuccess) return cuda_status(e);
    clamp_count_kernel<<<1, 1, 0, s>>>((const long long *)n_pairs_out, capacity, b.n_sort);
    // 3. keys into the tile buckets (cursors start at the bucket starts)
    e = cudaMemcpyAsync(b.tile_fill, b.tile_off, sizeof(uint32_t) * (size_t)T, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    const unsigned egrid = (unsigned)((m + kEmitRecs - 1) / kEmitRecs);
    bin_emit_kernel<<<egrid < 148u * 8u ? egrid : 148u * 8u, kBinThreads, 0, s>>>(
        vt, n, rec, tmax, opt->ellipse_cull, b.vis, b.counts + 2, b.tile_fill, b.n_sort, b.keys);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    // 4. sort every bucket; tile ranges
    seg_sort_small_kernel<<<grid_for(T * 32, 256), 256, 0, s>>>((uint32_t)T, b.tile_off, b.tile_cnt, b.n_sort,
                                                                 b.keys, pair_vals, tile_ranges, b.mid_list,
                                                                 b.counts, b.big_list, b.counts + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    e = launch_radix_buckets<128, kMidSeg>(b.mid_list, b.counts, b.tile_off, b.tile_cnt, b.keys, pair_vals,
                                          148 * 10, s);
    if (e != cudaSuccess) return cuda_status(e);
    // buckets above kMidSeg: the 4096-key and 8192-key radix CTAs, and
    // beyond that chunked passes through global memory (each kernel skips
    // the sizes it does not take)
    e = launch_radix_buckets<256, kSegMax>(b.big_list, b.counts + 1, b.tile_off, b.tile_cnt, b.keys, pair_vals,
                                          148 * 2, s);
    if (e != cudaSuccess) return cuda_status(e);
    e = launch_radix_buckets<512, kBigSeg, kSegMax>(b.big_list, b.counts + 1, b.tile_off, b.tile_cnt, b.keys,
                                                    pair_vals, 148, s);
    if (e != cudaSuccess) return cuda_status(e);
    {
        static bool huge_attr = false;
        const int smem = (int)sizeof(HugeSmem<256, kSegMax>);
        if (!huge_attr) {
            e = cudaFuncSetAttribute(seg_sort_huge_kernel<256, kSegMax>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return cuda_status(e);
            huge_attr = true;
        }
        seg_sort_huge_kernel<256, kSegMax><<<148 * 2, 256, smem, s>>>(b.big_list, b.counts + 1, b.tile_off,
                                                                        b.tile_cnt, b.keys, b.scratch, pair_vals,
                                                                        kBigSeg);
    }
    return cuda_status(cudaGetLastError());
}

#ifdef HM_CHECKED
namespace hm {
HM_CHECKED_READER(bin)
}  // namespace hm
#endif
