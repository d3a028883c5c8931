"""ctypes binding of libhm.so (the C ABI declared in include/hm.h).

Argument marshalling only: every function forwards to the entry point of the
same name.  Device buffers are passed as integer addresses (e.g.
``tensor.data_ptr()``), ``cams``/``opt`` as ctypes structures, the stream as
an integer ``cudaStream_t``.  Loading raises if the library has not been built
(``python -m paper_2506_06988_b300.build``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_float, c_int32, c_int64, c_size_t, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhm.so")
LIB_CHECKED_PATH = os.path.join(_HERE, "libhm_checked.so")

HM_OK = 0
HM_ERR_INVALID_ARG = 1
HM_ERR_CUDA = 2
HM_ERR_WORKSPACE = 3
HM_DEV_CAPACITY = 1
HM_DEV_TIMEOUT = 2
HM_DEV_BAD_INDEX = 4
HM_MAX_VIEWS = 32
HM_MAX_PAIRS = 0x3FFFFFFF
HM_TEX_RGB8 = 0
HM_TEX_RGBF32 = 1
HM_SH_F32 = 0
HM_SH_F16 = 1
HM_BWD_TEXTURE = 1
HM_BWD_BLEND = 2
HM_BWD_PROJECT = 4
HM_BWD_NOALLOC_BYTES = 16 << 20

EXPORTS = [
    "hm_default_options", "hm_last_error", "hm_total_tiles",
    "hm_rasterize_mesh_workspace_size", "hm_rasterize_mesh",
    "hm_project_gaussians", "hm_mip_filter_3d",
    "hm_bin_sort_workspace_size", "hm_bin_sort",
    "hm_blend_forward",
    "hm_blend_backward_workspace_size", "hm_blend_backward", "hm_blend_backward_noalloc",
    "hm_default_loss_params", "hm_hybrid_loss_workspace_size", "hm_hybrid_loss", "hm_hybrid_loss_u8",
    "hm_decode_u8",
    "hm_default_prune_params", "hm_mesh_prune_workspace_size", "hm_mesh_prune",
    "hm_adam_update", "hm_adam_update_dev", "hm_adam_advance", "hm_activate", "hm_activate_backward",
    "hm_selftest_bounded_waits", "hm_checked_status",
]


class HmCamera(ctypes.Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float), ("width", c_int32), ("height", c_int32)]


class HmOptions(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("batch", c_int32),
                ("mesh_cull", c_int32), ("near_gauss", c_float), ("near_mesh", c_float),
                ("bg", c_float * 3), ("bwd_stages", c_int32), ("ellipse_cull", c_int32),
                ("kernel_2d", c_float), ("antialias", c_int32), ("persistent", c_int32)]


class HmLossParams(ctypes.Structure):
    _fields_ = [("lambda_ssim", c_float), ("lambda_t", c_float), ("k", c_float)]


class HmPruneParams(ctypes.Structure):
    _fields_ = [("alpha_normal", c_float), ("alpha_area", c_float), ("angle_deg", c_float),
                ("alpha_group", c_int32)]


class HmError(RuntimeError):
    pass


_lib = None
_CAM_P = POINTER(HmCamera)
_OPT_P = POINTER(HmOptions)
_PRUNE_P = POINTER(HmPruneParams)
_LOSS_P = POINTER(HmLossParams)

_SIGS = {
    "hm_default_options": (None, [_OPT_P]),
    "hm_last_error": (ctypes.c_char_p, []),
    "hm_total_tiles": (c_int64, [_CAM_P, c_int32, _OPT_P]),
    "hm_rasterize_mesh_workspace_size": (c_size_t, [_CAM_P, c_int32, c_int32, c_int32, c_int64, _OPT_P]),
    "hm_rasterize_mesh": (c_int32, [_CAM_P, c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_int32,
                                    c_void_p, c_int32, c_int32, c_int32, _OPT_P, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p,
                                    c_void_p, c_size_t, c_void_p]),
    "hm_project_gaussians": (c_int32, [_CAM_P, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_int32, c_int32, _OPT_P,
                                       c_void_p, c_void_p]),
    "hm_mip_filter_3d": (c_int32, [_CAM_P, c_int32, c_int32, c_void_p, c_float, c_float, c_void_p,
                                   c_void_p]),
    "hm_bin_sort_workspace_size": (c_size_t, [_CAM_P, c_int32, c_int32, c_int64, _OPT_P]),
    "hm_bin_sort": (c_int32, [_CAM_P, c_int32, c_int32, c_void_p, c_void_p, _OPT_P, c_void_p,
                              c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hm_blend_forward": (c_int32, [_CAM_P, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, _OPT_P, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p]),
    "hm_blend_backward_workspace_size": (c_size_t, [c_int32, c_int32]),
    "hm_blend_backward": (c_int32, [_CAM_P, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                    _OPT_P, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_size_t, c_void_p]),
    "hm_default_loss_params": (None, [_LOSS_P]),
    "hm_default_prune_params": (None, [_PRUNE_P]),
    "hm_adam_update": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_float, c_float, c_float,
                                 c_float, c_int32, c_void_p]),
    "hm_adam_update_dev": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_float, c_float, c_float,
                                     c_float, c_void_p, c_void_p, c_void_p]),
    "hm_adam_advance": (c_int32, [c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p]),
    "hm_activate": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "hm_selftest_bounded_waits": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "hm_checked_status": (c_int32, [POINTER(c_int32), c_int32]),
    "hm_activate_backward": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p]),
    "hm_mesh_prune_workspace_size": (c_size_t, [_CAM_P, c_int32, c_int32, c_int32]),
    "hm_mesh_prune": (c_int32, [_CAM_P, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p,
                                _PRUNE_P, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hm_hybrid_loss_workspace_size": (c_size_t, [_CAM_P, c_int32]),
    "hm_decode_u8": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p]),
    "hm_hybrid_loss": (c_int32, [_CAM_P, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 _LOSS_P, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hm_hybrid_loss_u8": (c_int32, [_CAM_P, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    _LOSS_P, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "hm_blend_backward_noalloc": (c_int32, [_CAM_P, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                            c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                            _OPT_P, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p]),
}


def _open(path):
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load():
    """Load libhm.so (raises HmError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise HmError(f"{LIB_PATH} not built: run `python -m paper_2506_06988_b300.build`")
        _lib = _open(LIB_PATH)
    return _lib


_checked = None


def load_checked():
    """The index-checked library libhm_checked.so (same entry points; every
    index a kernel reads from a device buffer is checked and a failure is
    reported by hm_checked_status instead of faulting).  ``use(lib)``
    routes this module's functions to it."""
    global _checked
    if _checked is None:
        if not os.path.exists(LIB_CHECKED_PATH):
            raise HmError(f"{LIB_CHECKED_PATH} not built: run `python -m paper_2506_06988_b300.build --checked`")
        _checked = _open(LIB_CHECKED_PATH)
    return _checked


def use(handle):
    """Route the entry points of this module to ``handle`` (``load()`` or
    ``load_checked()``); returns the handle in use before."""
    global _lib
    before = load()
    _lib = handle
    return before


def hm_checked_status(reset: bool = True) -> int:
    """HM_DEV_BAD_INDEX if a check of the checked library failed since the
    last reset, else 0 (HmError from the default library, which has none)."""
    v = c_int32(0)
    check(load().hm_checked_status(ctypes.byref(v), int(bool(reset))), "hm_checked_status")
    return int(v.value)


def check_device_status(st: int) -> int:
    """Raise HmError for the device status bits that invalidate a result
    (HM_DEV_TIMEOUT: a bounded wait gave up; HM_DEV_BAD_INDEX: a pair list
    held an out-of-range record index, so a placeholder record was used);
    returns ``st`` (HM_DEV_CAPACITY is the caller's to handle)."""
    if st & HM_DEV_TIMEOUT:
        raise HmError("a bounded device wait timed out (HM_DEV_TIMEOUT)")
    if st & HM_DEV_BAD_INDEX:
        raise HmError("a pair list held an out-of-range record index (HM_DEV_BAD_INDEX)")
    return st


def last_error() -> str:
    return load().hm_last_error().decode()


def check(status: int, what: str = ""):
    if status != HM_OK:
        raise HmError(f"{what}: status {status}: {last_error()}")


def cameras(cams) -> ctypes.Array:
    """Array of HmCamera from objects with R, t, fx, fy, cx, cy, width, height."""
    arr = (HmCamera * len(cams))()
    for k, c in enumerate(cams):
        arr[k].R[:] = [float(x) for x in c.R.reshape(9)]
        arr[k].t[:] = [float(x) for x in c.t.reshape(3)]
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[k].width, arr[k].height = int(c.width), int(c.height)
    return arr


def options(tile=(16, 16), batch=None, mesh_cull=True, bg=(0.0, 0.0, 0.0), near_gauss=0.2,
            near_mesh=0.01, ellipse_cull=True, mip=False, persistent=False) -> HmOptions:
    """hm_options; ``mip`` selects Mip-Splatting's 2D Mip filter (kernel 0.1
    with opacity compensation) instead of the 3DGS 0.3 dilation; with
    ``persistent`` the blend kernels claim (view, tile) work from a counter.
    The staging batch defaults to 128 list entries (the tile's pixel count
    if smaller)."""
    o = HmOptions()
    load().hm_default_options(ctypes.byref(o))
    o.persistent = int(bool(persistent))
    if mip:
        o.kernel_2d, o.antialias = 0.1, 1
    o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
    o.batch = int(batch) if batch is not None else min(128, int(tile[0] * tile[1]))
    o.mesh_cull = int(bool(mesh_cull))
    o.ellipse_cull = int(bool(ellipse_cull))
    o.near_gauss, o.near_mesh = float(near_gauss), float(near_mesh)
    o.bg[:] = [float(x) for x in bg]
    return o


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


# ---- entry points (same names as the C ABI) ---------------------------------

def hm_total_tiles(cams, opt) -> int:
    return load().hm_total_tiles(cams, len(cams), ctypes.byref(opt))


def hm_rasterize_mesh_workspace_size(cams, n_verts, n_faces, item_capacity, opt) -> int:
    return load().hm_rasterize_mesh_workspace_size(cams, len(cams), n_verts, n_faces, item_capacity,
                                                   ctypes.byref(opt))


def hm_rasterize_mesh(cams, verts, uvs, n_verts, faces, n_faces, tex, tex_w, tex_h, tex_format,
                      opt, tri_id, depth, rgb, uv, tile_max_depth, item_capacity, n_items_out,
                      d_status, ws, ws_bytes, stream):
    return load().hm_rasterize_mesh(cams, len(cams), _ptr(verts), _ptr(uvs), n_verts, _ptr(faces),
                                    n_faces, _ptr(tex), tex_w, tex_h, tex_format, ctypes.byref(opt),
                                    _ptr(tri_id), _ptr(depth), _ptr(rgb), _ptr(uv),
                                    _ptr(tile_max_depth), item_capacity, _ptr(n_items_out),
                                    _ptr(d_status), _ptr(ws), ws_bytes, stream)


def hm_project_gaussians(cams, n, means, scales, quats, opacity, sh, sh_degree, sh_format, opt,
                         records, stream, filter_3d=None):
    return load().hm_project_gaussians(cams, len(cams), n, _ptr(means), _ptr(scales), _ptr(quats),
                                       _ptr(opacity), _ptr(filter_3d), _ptr(sh), sh_degree, sh_format,
                                       ctypes.byref(opt), _ptr(records), stream)


def hm_mip_filter_3d(cams, n, means, s2, near_z, filter_3d, stream):
    return load().hm_mip_filter_3d(cams, len(cams), n, _ptr(means), s2, near_z, _ptr(filter_3d), stream)


def hm_bin_sort_workspace_size(cams, n, capacity, opt) -> int:
    return load().hm_bin_sort_workspace_size(cams, len(cams), n, capacity, ctypes.byref(opt))


def hm_bin_sort(cams, n, records, tile_max_depth, opt, pair_vals, capacity, n_pairs_out,
                tile_ranges, d_status, ws, ws_bytes, stream):
    return load().hm_bin_sort(cams, len(cams), n, _ptr(records), _ptr(tile_max_depth),
                              ctypes.byref(opt), _ptr(pair_vals), capacity, _ptr(n_pairs_out),
                              _ptr(tile_ranges), _ptr(d_status), _ptr(ws), ws_bytes, stream)


def hm_blend_forward(cams, n, records, pair_vals, tile_ranges, mesh_depth, mesh_rgb, opt, out_rgb,
                     out_T, n_contrib, last_idx, eval_stats, d_status, stream, work=None):
    return load().hm_blend_forward(cams, len(cams), n, _ptr(records), _ptr(pair_vals),
                                   _ptr(tile_ranges), _ptr(mesh_depth), _ptr(mesh_rgb),
                                   ctypes.byref(opt), _ptr(out_rgb), _ptr(out_T), _ptr(n_contrib),
                                   _ptr(last_idx), _ptr(eval_stats), _ptr(d_status), _ptr(work), stream)


def hm_blend_backward_workspace_size(n_views, n) -> int:
    return load().hm_blend_backward_workspace_size(n_views, n)


def hm_blend_backward(cams, n, means, scales, quats, opacity, sh, sh_degree, sh_format, records,
                      pair_vals, tile_ranges, mesh_depth, mesh_rgb, mesh_uv, tex_w, tex_h, opt,
                      out_T, last_idx, dL_drgb, dL_dT, d_means, d_scales, d_quats, d_opacity, d_sh,
                      d_tex, d_status, ws, ws_bytes, stream, dL_dmesh=None, filter_3d=None):
    return load().hm_blend_backward(cams, len(cams), n, _ptr(means), _ptr(scales), _ptr(quats),
                                    _ptr(opacity), _ptr(filter_3d), _ptr(sh), sh_degree, sh_format,
                                    _ptr(records),
                                    _ptr(pair_vals), _ptr(tile_ranges), _ptr(mesh_depth),
                                    _ptr(mesh_rgb), _ptr(mesh_uv), tex_w, tex_h, ctypes.byref(opt),
                                    _ptr(out_T), _ptr(last_idx), _ptr(dL_drgb), _ptr(dL_dT),
                                    _ptr(dL_dmesh), _ptr(d_means), _ptr(d_scales), _ptr(d_quats),
                                    _ptr(d_opacity), _ptr(d_sh), _ptr(d_tex), _ptr(d_status), _ptr(ws),
                                    ws_bytes, stream)


def hm_blend_backward_noalloc(cams, n, means, scales, quats, opacity, sh, sh_degree, sh_format,
                              records, pair_vals, tile_ranges, mesh_depth, mesh_rgb, mesh_uv, tex_w,
                              tex_h, opt, out_T, last_idx, dL_drgb, dL_dT, d_means, d_scales, d_quats,
                              d_opacity, d_sh, d_tex, d_status, stream, filter_3d=None, dL_dmesh=None):
    """hm_blend_backward without a workspace argument: the scratch is the
    library's static 16 MiB device array (for callers that cannot allocate)."""
    return load().hm_blend_backward_noalloc(cams, len(cams), n, _ptr(means), _ptr(scales),
                                            _ptr(quats), _ptr(opacity), _ptr(filter_3d), _ptr(sh),
                                            sh_degree,
                                            sh_format, _ptr(records), _ptr(pair_vals),
                                            _ptr(tile_ranges), _ptr(mesh_depth), _ptr(mesh_rgb),
                                            _ptr(mesh_uv), tex_w, tex_h, ctypes.byref(opt),
                                            _ptr(out_T), _ptr(last_idx), _ptr(dL_drgb), _ptr(dL_dT),
                                            _ptr(dL_dmesh), _ptr(d_means), _ptr(d_scales), _ptr(d_quats),
                                            _ptr(d_opacity), _ptr(d_sh), _ptr(d_tex),
                                            _ptr(d_status), stream)


HM_PRUNE_NORMAL, HM_PRUNE_ANGLE, HM_PRUNE_AREA, HM_PRUNE_GROUP = 1, 2, 4, 8


def prune_params(alpha_normal=None, alpha_area=None, angle_deg=None, alpha_group=None) -> HmPruneParams:
    p = HmPruneParams()
    load().hm_default_prune_params(ctypes.byref(p))
    for k, v in (("alpha_normal", alpha_normal), ("alpha_area", alpha_area), ("angle_deg", angle_deg),
                 ("alpha_group", alpha_group)):
        if v is not None:
            setattr(p, k, v)
    return p


def hm_mesh_prune_workspace_size(cams, n_verts, n_faces) -> int:
    return load().hm_mesh_prune_workspace_size(cams, len(cams) if cams is not None else 0, n_verts, n_faces)


def hm_mesh_prune(cams, verts, n_verts, faces, n_faces, tri_id, normals, params, flags, label, ws, ws_bytes,
                  stream):
    return load().hm_mesh_prune(cams, len(cams) if cams is not None else 0, _ptr(verts), n_verts, _ptr(faces),
                                n_faces, _ptr(tri_id), _ptr(normals), ctypes.byref(params), _ptr(flags),
                                _ptr(label), _ptr(ws), ws_bytes, stream)


def hm_adam_update(param, grad, m, v, n, lr, beta1, beta2, eps, step, stream):
    return load().hm_adam_update(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), n, lr, beta1, beta2, eps, step,
                                 stream)


def hm_adam_update_dev(param, grad, m, v, n, lr, beta1, beta2, eps, d_rc, d_status, stream):
    return load().hm_adam_update_dev(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), n, lr, beta1, beta2, eps,
                                     _ptr(d_rc), _ptr(d_status), stream)


def hm_adam_advance(d_step, beta1, beta2, d_rc, d_status, stream):
    return load().hm_adam_advance(_ptr(d_step), beta1, beta2, _ptr(d_rc), _ptr(d_status), stream)


def hm_selftest_bounded_waits(d_zero_slot, d_status, d_out, stream):
    return load().hm_selftest_bounded_waits(_ptr(d_zero_slot), _ptr(d_status), _ptr(d_out), stream)


def hm_activate(n, log_scales, logit, scales, opacity, stream):
    return load().hm_activate(n, _ptr(log_scales), _ptr(logit), _ptr(scales), _ptr(opacity), stream)


def hm_activate_backward(n, scales, opacity, d_scales, d_opacity, d_log_scales, d_logit, stream):
    return load().hm_activate_backward(n, _ptr(scales), _ptr(opacity), _ptr(d_scales), _ptr(d_opacity),
                                       _ptr(d_log_scales), _ptr(d_logit), stream)


def loss_params(lambda_ssim=None, lambda_t=None, k=None) -> HmLossParams:
    p = HmLossParams()
    load().hm_default_loss_params(ctypes.byref(p))
    if lambda_ssim is not None:
        p.lambda_ssim = float(lambda_ssim)
    if lambda_t is not None:
        p.lambda_t = float(lambda_t)
    if k is not None:
        p.k = float(k)
    return p


def hm_decode_u8(src, n, dst, stream):
    return load().hm_decode_u8(_ptr(src), n, _ptr(dst), stream)


def hm_hybrid_loss_workspace_size(cams) -> int:
    return load().hm_hybrid_loss_workspace_size(cams, len(cams))


def hm_hybrid_loss(cams, out_rgb, target, mesh_rgb, out_T, mesh_depth, params, loss_out, dL_drgb,
                   dL_dmesh, ws, ws_bytes, stream):
    return load().hm_hybrid_loss(cams, len(cams), _ptr(out_rgb), _ptr(target), _ptr(mesh_rgb), _ptr(out_T),
                                 _ptr(mesh_depth), ctypes.byref(params), _ptr(loss_out), _ptr(dL_drgb),
                                 _ptr(dL_dmesh), _ptr(ws), ws_bytes, stream)


def hm_hybrid_loss_u8(cams, out_rgb, target, mesh_rgb, out_T, mesh_depth, params, loss_out, dL_drgb,
                      dL_dmesh, ws, ws_bytes, stream):
    return load().hm_hybrid_loss_u8(cams, len(cams), _ptr(out_rgb), _ptr(target), _ptr(mesh_rgb),
                                    _ptr(out_T), _ptr(mesh_depth), ctypes.byref(params), _ptr(loss_out),
                                    _ptr(dL_drgb), _ptr(dL_dmesh), _ptr(ws), ws_bytes, stream)
