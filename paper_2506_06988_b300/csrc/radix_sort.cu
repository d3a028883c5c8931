// radix_sort.cu -- stable LSD radix sort of uint32 (key, value) pairs,
// 8-bit digits, one "onesweep" pass per digit.
//
// A histogram kernel counts every digit of every pass in one read of the
// keys.  Each pass then ranks a tile of 4096 keys per CTA (warp-level
// match.any ranking keeps the input order among equal digits, which makes the
// sort stable), obtains the tile's per-digit offset from its predecessors
// through a decoupled look-back (bounded waits), reorders the tile in shared
// memory and writes every digit's run with coalesced stores.
//
// The CTAs are persistent: each loops taking tile tickets from an atomic
// counter until the tiles run out, so the grid never exceeds one wave and
// the element count can live in device memory (graph-capturable, no host
// round trip).  A ticket is only taken by a running CTA, so every tile a
// look-back waits on is being processed: the waits terminate.
#include "hm_internal.cuh"

namespace hm {

namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr uint32_t kLbAgg = 1u << 30;
constexpr uint32_t kLbInc = 2u << 30;
constexpr uint32_t kLbMask = (1u << 30) - 1;

__global__ void __launch_bounds__(256)
radix_hist_kernel(const uint32_t *__restrict__ keys, const long long *n_dev, int passes,
                  uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_hist[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const long long n = *n_dev;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

struct PassSmem {
    uint32_t whist[kWarps][257];   // per-warp running digit counts, then warp offsets
    uint32_t dstart[257];          // tile-local start of each digit
    uint32_t gofs[256];            // global position of the tile's first element of each digit
    uint32_t gbase[256];           // exclusive scan of the global digit histogram
    uint32_t keys[kSortTile];
    uint32_t vals[kSortTile];
    unsigned int tile;
};

__global__ void __launch_bounds__(kSortThreads)
onesweep_kernel(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, const long long *n_dev,
                int shift, const uint32_t *__restrict__ ghist, uint32_t *lookback,
                unsigned int *ticket, int32_t *d_status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PassSmem &S = *reinterpret_cast<PassSmem *>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long n = *n_dev;
    const long long ntiles = (n + kSortTile - 1) / kSortTile;

    // exclusive scan of this pass's global digit histogram (thread t = digit t)
    {
        uint32_t c = ghist[t];
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.dstart[warp] = incl;
        __syncthreads();
        uint32_t woff = 0;
        for (int w = 0; w < warp; ++w) woff += S.dstart[w];
        S.gbase[t] = woff + incl - c;
        __syncthreads();
    }

    for (;;) {
        if (t == 0) S.tile = atomicAdd(ticket, 1u);
        for (int i = t; i < kWarps * 257; i += kSortThreads) (&S.whist[0][0])[i] = 0;
        __syncthreads();
        const long long tile = S.tile;
        if (tile >= ntiles) break;
        const long long base = tile * kSortTile;

        // ---- load (warp-contiguous chunks of 512) and rank within the warp
        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        int dig[kSortItems];
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            long long e = base + (long long)warp * (32 * kSortItems) + j * 32 + lane;
            bool valid = e < n;
            key[j] = valid ? kin[e] : 0xFFFFFFFFu;
            val[j] = valid ? (vin ? vin[e] : (uint32_t)e) : 0u;
            int d = valid ? (int)((key[j] >> shift) & 255u) : 256;
            dig[j] = d;
            uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t before = S.whist[warp][d];
            __syncwarp();
            if ((peers & lt) == 0) S.whist[warp][d] = before + __popc(peers);
            __syncwarp();
            rank[j] = before + __popc(peers & lt);
        }
        __syncthreads();

        // ---- per digit (thread t = digit t): warp offsets, tile count
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = S.whist[w][t];
            S.whist[w][t] = cnt;
            cnt += c;
        }
        // tile-local digit starts: exclusive scan of cnt over digits
        {
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            __shared__ uint32_t s_w[kWarps];
            if (lane == 31) s_w[warp] = incl;
            __syncthreads();
            uint32_t woff = 0;
            for (int w = 0; w < warp; ++w) woff += s_w[w];
            S.dstart[t] = woff + incl - cnt;
            if (t == 0) S.dstart[256] = 0;
        }
        // ---- decoupled look-back for digit t
        {
            uint32_t *lb = lookback + tile * 256;
            uint32_t prefix = 0;
            if (tile == 0) {
                st_volatile_u32(&lb[t], kLbInc | cnt);
            } else {
                st_volatile_u32(&lb[t], kLbAgg | cnt);
                long long p = tile - 1;
                int spins = 0;
                while (p >= 0) {
                    uint32_t s = ld_volatile_u32(lookback + p * 256 + t);
                    uint32_t f = s >> 30;
                    if (f == 0) {
                        if (++spins > kSpinLimit) {
                            set_status(d_status, HM_DEV_TIMEOUT);
                            break;
                        }
                        __nanosleep(64);
                        continue;
                    }
                    prefix += s & kLbMask;
                    if (f == 2) break;
                    --p;
                }
                st_volatile_u32(&lb[t], kLbInc | (prefix + cnt));
            }
            S.gofs[t] = S.gbase[t] + prefix;
        }
        __syncthreads();

        // ---- reorder the tile in shared memory (digit-major, stable)
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            int d = dig[j];
            if (d < 256) {
                uint32_t pos = S.dstart[d] + S.whist[warp][d] + rank[j];
                S.keys[pos] = key[j];
                S.vals[pos] = val[j];
            }
        }
        __syncthreads();
        const int tcount = (int)min((long long)kSortTile, n - base);
#pragma unroll 4
        for (int i = t; i < tcount; i += kSortThreads) {
            uint32_t k = S.keys[i];
            int d = (int)((k >> shift) & 255u);
            uint32_t g = S.gofs[d] + (uint32_t)(i - (int)S.dstart[d]);
            kout[g] = k;
            vout[g] = S.vals[i];
        }
        __syncthreads();
    }
}

int g_sort_blocks = 0;

}  // namespace

cudaError_t launch_radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                              const long long *n_dev, long long n_max, int passes,
                              bool identity_vals, int32_t *d_status, SortWs ws, cudaStream_t s) {
    if (passes <= 0 || n_max <= 0) return cudaSuccess;
    const size_t smem = sizeof(PassSmem);
    if (g_sort_blocks == 0) {
        cudaError_t e = cudaFuncSetAttribute(onesweep_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_kernel, kSortThreads, smem);
        g_sort_blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    cudaError_t e = cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * 4 * 256, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned int) * 4, s);
    if (e != cudaSuccess) return e;
    const long long need_tiles = sort_tiles(n_max) + 1;
    for (int p = 0; p < passes; ++p) {
        e = cudaMemsetAsync(ws.lookback + (size_t)256 * ws.max_tiles * p, 0,
                            sizeof(uint32_t) * 256 * (size_t)need_tiles, s);
        if (e != cudaSuccess) return e;
    }
    long long hblocks = (n_max + 255) / 256;
    if (hblocks > 4 * (long long)g_sort_blocks) hblocks = 4 * (long long)g_sort_blocks;
    radix_hist_kernel<<<(unsigned)hblocks, 256, 0, s>>>(k0, n_dev, passes, ws.hist);
    long long maxt = sort_tiles(n_max);
    unsigned grid = (unsigned)(maxt < g_sort_blocks ? maxt : g_sort_blocks);
    for (int p = 0; p < passes; ++p) {
        const uint32_t *kin = (p & 1) ? k1 : k0;
        const uint32_t *vin = (p & 1) ? v1 : v0;
        uint32_t *kout = (p & 1) ? k0 : k1;
        uint32_t *vout = (p & 1) ? v0 : v1;
        if (p == 0 && identity_vals) vin = nullptr;   // values = input positions
        onesweep_kernel<<<grid, kSortThreads, smem, s>>>(kin, vin, kout, vout, n_dev, 8 * p,
                                                          ws.hist + 256 * p,
                                                          ws.lookback + (size_t)256 * ws.max_tiles * p,
                                                          ws.ticket + p, d_status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hm
