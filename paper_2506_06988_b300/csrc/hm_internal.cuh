// hm_internal.cuh -- device-side types and helpers shared by the kernels of
// libhm (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "hm.h"

namespace hm {

// ---------------------------------------------------------------------------
// per-camera constants, passed by value in kernel parameter space
// ---------------------------------------------------------------------------
struct ViewDev {
    float R[9];
    float t[3];
    float campos[3];       // camera centre -R^T t (world)
    float fx, fy, cx, cy;
    int W, H, tiles_x, tiles_y;
    int tile_off;          // first global tile id of this camera
    int pad;
    long long pix_off;     // first global pixel of this camera
};

struct ViewTable {
    int n_views, tile_w, tile_h, total_tiles;
    long long total_pixels;
    ViewDev v[HM_MAX_VIEWS];
};

// camera owning global tile `gt` (tile_off is increasing)
// Screen-space kernel and the Mip-Splatting filters (see hm_options and
// hm_project_gaussians): f3d the per-Gaussian 3D smoothing variance or null,
// kernel the variance added to the projected covariance, antialias the 2D
// Mip filter's opacity compensation.
struct Filters {
    const float *f3d;
    float kernel;
    int antialias;
};

__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int gt) {
    int v = 0;
    for (int k = 1; k < vt.n_views; ++k)
        if (vt.v[k].tile_off <= gt) v = k;
    return v;
}

__device__ __forceinline__ int view_of_pixel(const ViewTable &vt, long long gp) {
    int v = 0;
    for (int k = 1; k < vt.n_views; ++k)
        if (vt.v[k].pix_off <= gp) v = k;
    return v;
}

// ---------------------------------------------------------------------------
// projected Gaussian record (48 bytes)
//   a = {mean_x, mean_y, K conic_xx, 2K conic_xy}
//   b = {K conic_yy, opacity, depth, tile x-range (u16 x0 | u16 x1 << 16)}
//   c = {r, g, b, tile y-range (u16 y0 | u16 y1 << 16)}
// with K = -log2(e)/2, so that the blend's exponent is q = K d^2 and
// exp(-d^2/2) = 2^q with no per-pixel scaling; the blend kernels copy
// records into shared memory unchanged.  An empty range has x0 > x1.
// ---------------------------------------------------------------------------
constexpr float kConicScale = -0.72134752044448170f;   // K = -log2(e)/2

struct __align__(16) Record {
    float4 a, b, c;
};
static_assert(sizeof(Record) == 48, "record layout");

__host__ __device__ __forceinline__ uint32_t pack_range(uint32_t lo, uint32_t hi) {
    return (lo & 0xFFFFu) | (hi << 16);
}
__host__ __device__ __forceinline__ void unpack_range(uint32_t r, int &lo, int &hi) {
    lo = (int)(r & 0xFFFFu);
    hi = (int)(r >> 16);
}
constexpr uint32_t kEmptyRange = 0x0000FFFFu;   // lo = 65535 > hi = 0

// ---------------------------------------------------------------------------
// status words and bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t *st, int32_t bit) {
    if (st) atomicOr(st, bit);
}

// polls of a not-yet-published predecessor before a wait gives up (each poll
// sleeps ~100 ns, so the bound is several hundred milliseconds)
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_volatile_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_volatile_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Bounded wait for a decoupled look-back slot to be published (its top two
// bits nonzero): false after kSpinLimit polls, with HM_DEV_TIMEOUT set.
__device__ __forceinline__ bool wait_published(const unsigned long long *slot, unsigned long long &val,
                                               int32_t *d_status) {
    for (int spins = 0;; ++spins) {
        val = ld_volatile_u64(slot);
        if ((val >> 62) != 0) return true;
        if (spins >= kSpinLimit) {
            set_status(d_status, HM_DEV_TIMEOUT);
            return false;
        }
        __nanosleep(100);
    }
}

// ---------------------------------------------------------------------------
// Checked build (HM_CHECKED defined: libhm_checked.so).  Every index a
// kernel reads from a device buffer -- list entries, bucket and range
// bounds, tile ids, slots -- is checked against the bound it must respect
// before it is used; a failed check sets a bit in this translation unit's
// checked-status word (read and cleared by hm_checked_status) and the access
// is skipped, so a corrupt list is reported instead of faulting.  In the
// default build hm_check is the constant true and the checks compile away.
// ---------------------------------------------------------------------------
#ifdef HM_CHECKED
static __device__ int g_hm_checked_bad;
__device__ __forceinline__ bool hm_check(bool ok) {
    if (!ok) atomicOr(&g_hm_checked_bad, 1);
    return ok;
}
// defines the host reader of this translation unit's word
#define HM_CHECKED_READER(name)                                                     \
    int hm_checked_read_##name(bool reset) {                                       \
        int v = 0;                                                                  \
        if (cudaMemcpyFromSymbol(&v, g_hm_checked_bad, sizeof(int)) != cudaSuccess) \
            return -1;                                                              \
        if (reset) {                                                                \
            const int z = 0;                                                        \
            if (cudaMemcpyToSymbol(g_hm_checked_bad, &z, sizeof(int)) != cudaSuccess)  \
                return -1;                                                          \
        }                                                                           \
        return v;                                                                   \
    }
#else
__device__ __forceinline__ constexpr bool hm_check(bool) { return true; }
#define HM_CHECKED_READER(name)
#endif

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// host launchers (one per .cu file)
// ---------------------------------------------------------------------------
struct ScanWs {
    unsigned long long *tile_status;   // [max_tiles]
    unsigned int *ticket;              // [1]
};
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
inline long long scan_tiles(long long n) { return (n + kScanTile - 1) / kScanTile; }

// out[i] = sum_{j<i} in[idx ? idx[j] : j] (uint32, exclusive); *total (int64)
// = the full sum; if capacity >= 0 and the sum exceeds it, HM_DEV_CAPACITY.
// The element count is n, or *n_dev (<= n) when n_dev is given.
cudaError_t launch_scan(const uint32_t *in, const uint32_t *idx, uint32_t *out, long long n,
                        long long *total, long long capacity, int32_t *d_status, ScanWs ws,
                        cudaStream_t s, const long long *n_dev = nullptr);

cudaError_t launch_fill_i64(long long *p, long long v, cudaStream_t s);

}  // namespace hm
