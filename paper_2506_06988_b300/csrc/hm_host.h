// hm_host.h -- host-side helpers shared by the C-ABI entry points.
#pragma once

#include <cuda_runtime.h>

#include "hm.h"
#include "hm_internal.cuh"

namespace hm {

// Record the thread-local error text and return `code`.
hm_status fail(hm_status code, const char *fmt, ...);
// HM_OK, or HM_ERR_CUDA with the CUDA error text recorded.
hm_status cuda_status(cudaError_t e);
// Validate cameras and options and fill the by-value view table.
bool build_view_table(const hm_camera *cams, int n_views, const hm_options *opt, ViewTable *vt);
bool tile_shape_ok(int tw, int th);
#ifdef HM_CHECKED
// checked build: the checked-status words of the translation units with
// index checks (-1 if the read failed); `reset` clears them
int hm_checked_read_mesh(bool reset);
int hm_checked_read_bin(bool reset);
int hm_checked_read_blend_fwd(bool reset);
int hm_checked_read_blend_bwd(bool reset);
#endif

// bump allocator over a caller workspace (256-byte aligned sub-buffers)
struct WsCarver {
    char *base;
    size_t off = 0;
    explicit WsCarver(void *p) : base((char *)p) {}
    template <class T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * count;
        return p;
    }
};

}  // namespace hm
