// scan.cu -- single-pass device-wide exclusive scan (decoupled look-back).
//
// Each CTA scans a tile of 4096 uint32 values, publishes its aggregate, then
// looks back over its predecessors' published prefixes.  Tiles are handed
// out through an atomic ticket, so every predecessor of a CTA's tile belongs
// to a CTA that is already running: the look-back always terminates.  Each
// wait is still bounded; on expiry HM_DEV_TIMEOUT is set and the CTA
// proceeds with what it has.
#include "hm_host.h"
#include "hm_internal.cuh"
#include "tma.cuh"

namespace hm {

namespace {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__global__ void __launch_bounds__(kScanThreads)
scan_kernel(const uint32_t *__restrict__ in, const uint32_t *__restrict__ idx,
            uint32_t *__restrict__ out, long long n_host, const long long *n_dev, long long *total,
            long long capacity, int32_t *d_status, unsigned long long *tstat, unsigned int *ticket) {
    __shared__ uint32_t s_buf[kScanTile];
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned int s_tile;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long n = n_dev ? *n_dev : n_host;
    if (t == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    const long long base = tile * kScanTile;
    if (base >= n) {
        // beyond the element count (count held on the device): nothing to do;
        // an empty input still reports a zero total
        if (t == 0 && tile == 0 && total) *total = 0;
        return;
    }

    // striped (coalesced) load into shared memory
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        long long e = base + j * kScanThreads + t;
        uint32_t v = 0;
        if (e < n) v = idx ? in[idx[e]] : in[e];
        s_buf[j * kScanThreads + t] = v;
    }
    __syncthreads();
    // blocked read: thread t owns elements [t*16, t*16+16)
    uint32_t loc[kScanItems];
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        loc[j] = s_buf[t * kScanItems + j];
        sum += loc[j];
    }
    // block exclusive scan of the thread sums
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = wi - w;   // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) {
            // lane 7 holds the tile aggregate in wi: publish and look back
            unsigned long long agg = wi;
            unsigned long long prefix = 0;
            if (tile == 0) {
                st_volatile_u64(&tstat[0], kFlagInc | agg);
            } else {
                st_volatile_u64(&tstat[tile], kFlagAgg | agg);
                long long p = tile - 1;
                while (p >= 0) {
                    unsigned long long s;
                    if (!wait_published(&tstat[p], s, d_status)) break;
                    prefix += s & kValMask;
                    if ((s >> 62) == 2) break;
                    --p;
                }
                st_volatile_u64(&tstat[tile], kFlagInc | (prefix + agg));
            }
            s_prefix = prefix;
            if (base + kScanTile >= n) {
                long long tot = (long long)(prefix + agg);
                if (total) *total = tot;
                if (capacity >= 0 && tot > capacity) set_status(d_status, HM_DEV_CAPACITY);
            }
        }
    }
    __syncthreads();
    unsigned long long run = s_prefix + s_warp[warp] + (incl - sum);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        s_buf[t * kScanItems + j] = (uint32_t)run;
        run += loc[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        long long e = base + j * kScanThreads + t;
        if (e < n) out[e] = s_buf[j * kScanThreads + t];
    }
}

__global__ void fill_i64_kernel(long long *p, long long v) { *p = v; }

}  // namespace

cudaError_t launch_fill_i64(long long *p, long long v, cudaStream_t s) {
    fill_i64_kernel<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *in, const uint32_t *idx, uint32_t *out, long long n,
                        long long *total, long long capacity, int32_t *d_status, ScanWs ws,
                        cudaStream_t s, const long long *n_dev) {
    long long tiles = scan_tiles(n);
    cudaError_t e = cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (n <= 0) {
        if (total) e = cudaMemsetAsync(total, 0, sizeof(long long), s);
        return e;
    }
    e = cudaMemsetAsync(ws.tile_status, 0, sizeof(unsigned long long) * tiles, s);
    if (e != cudaSuccess) return e;
    scan_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, idx, out, n, n_dev, total, capacity,
                                                         d_status, ws.tile_status, ws.ticket);
    return cudaGetLastError();
}

}  // namespace hm

namespace hm {
namespace {

// The failure-detection self-test: the library's two bounded waits, each on
// something nothing completes -- a look-back slot never published and an
// mbarrier nobody arrives at -- must give up, report HM_DEV_TIMEOUT and return.
__global__ void selftest_waits_kernel(const unsigned long long *never, int32_t *d_status, int32_t *out) {
    __shared__ uint64_t bar;
    unsigned long long v = 0;
    const bool got_slot = wait_published(never, v, d_status);
    mbar_init(&bar, 1);
    mbar_fence_init();
    const bool got_bar = mbar_wait(&bar, 0);
    if (!got_bar) set_status(d_status, HM_DEV_TIMEOUT);
    mbar_inval(&bar);
    out[0] = got_slot ? 1 : 0;
    out[1] = got_bar ? 1 : 0;
}

}  // namespace
}  // namespace hm

extern "C" hm_status hm_selftest_bounded_waits(const unsigned long long *d_zero_slot, int32_t *d_status,
                                               int32_t *d_out, void *stream) {
    if (!d_zero_slot || !d_status || !d_out) return hm::fail(HM_ERR_INVALID_ARG, "null pointer");
    hm::selftest_waits_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_zero_slot, d_status, d_out);
    return hm::cuda_status(cudaGetLastError());
}
