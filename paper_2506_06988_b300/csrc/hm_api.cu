// hm_api.cu -- shared pieces of the C ABI: options, error text, camera table.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "hm_host.h"

namespace hm {

static thread_local char g_err[512] = "";

hm_status fail(hm_status code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

hm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return HM_OK;
    return fail(HM_ERR_CUDA, "CUDA error %d: %s", (int)e, cudaGetErrorString(e));
}

bool tile_shape_ok(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 32 && th == 8) || (tw == 8 && th == 8);
}

bool build_view_table(const hm_camera *cams, int n_views, const hm_options *opt, ViewTable *vt) {
    if (!cams || !opt) { fail(HM_ERR_INVALID_ARG, "null cams or opt"); return false; }
    if (n_views < 1 || n_views > HM_MAX_VIEWS) {
        fail(HM_ERR_INVALID_ARG, "n_views must be in 1..%d", HM_MAX_VIEWS);
        return false;
    }
    if (!tile_shape_ok(opt->tile_w, opt->tile_h)) {
        fail(HM_ERR_INVALID_ARG, "tile shape %dx%d not in {16x16, 32x8, 8x8}", opt->tile_w, opt->tile_h);
        return false;
    }
    memset(vt, 0, sizeof(*vt));
    vt->n_views = n_views;
    vt->tile_w = opt->tile_w;
    vt->tile_h = opt->tile_h;
    long long tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const hm_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384) {
            fail(HM_ERR_INVALID_ARG, "camera %d: image size %dx%d out of range", v, c.width, c.height);
            return false;
        }
        if (!(c.fx > 0.f) || !(c.fy > 0.f)) {
            fail(HM_ERR_INVALID_ARG, "camera %d: focal lengths must be positive", v);
            return false;
        }
        ViewDev &d = vt->v[v];
        memcpy(d.R, c.R, sizeof(d.R));
        memcpy(d.t, c.t, sizeof(d.t));
        for (int j = 0; j < 3; ++j)
            d.campos[j] = (float)(-((double)c.R[j] * c.t[0] + (double)c.R[3 + j] * c.t[1] +
                                    (double)c.R[6 + j] * c.t[2]));
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        d.W = c.width;
        d.H = c.height;
        d.tiles_x = (c.width + opt->tile_w - 1) / opt->tile_w;
        d.tiles_y = (c.height + opt->tile_h - 1) / opt->tile_h;
        d.tile_off = (int)tiles;
        d.pix_off = pix;
        tiles += (long long)d.tiles_x * d.tiles_y;
        pix += (long long)c.width * c.height;
    }
    if (tiles >= (1ll << 24)) { fail(HM_ERR_INVALID_ARG, "too many tiles (%lld)", tiles); return false; }
    vt->total_tiles = (int)tiles;
    vt->total_pixels = pix;
    return true;
}

}  // namespace hm

using namespace hm;

extern "C" void hm_default_options(hm_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->tile_w = 16;
    opt->tile_h = 16;
    opt->batch = 128;
    opt->mesh_cull = 1;
    opt->near_gauss = 0.2f;
    opt->near_mesh = 0.01f;
    opt->bwd_stages = 0;
    opt->ellipse_cull = 1;
    opt->kernel_2d = 0.3f;
    opt->antialias = 0;
}

extern "C" const char *hm_last_error(void) { return g_err; }

extern "C" int64_t hm_total_tiles(const hm_camera *cams, int32_t n_views, const hm_options *opt) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt)) return -1;
    return vt.total_tiles;
}

extern "C" hm_status hm_checked_status(int32_t *bits, int32_t reset) {
    if (!bits) return fail(HM_ERR_INVALID_ARG, "null pointer");
#ifdef HM_CHECKED
    const int r[4] = {hm_checked_read_mesh(reset != 0), hm_checked_read_bin(reset != 0),
                      hm_checked_read_blend_fwd(reset != 0), hm_checked_read_blend_bwd(reset != 0)};
    int v = 0;
    for (int k = 0; k < 4; ++k) {
        if (r[k] < 0) return fail(HM_ERR_CUDA, "reading the checked-status words failed");
        v |= r[k];
    }
    *bits = v ? HM_DEV_BAD_INDEX : 0;
    return HM_OK;
#else
    (void)reset;
    *bits = 0;
    return fail(HM_ERR_INVALID_ARG, "not the checked build (libhm_checked.so)");
#endif
}
