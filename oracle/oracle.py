"""Python front end of the CPU FP64 oracle (``hm_oracle.c``).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, the smoke check and the
benchmark's CPU-baseline leg.  It never imports the CUDA package; inputs are
plain numpy arrays or duck-typed objects with the attributes of the scene
generator's ``Camera``/``Gaussians``/``Mesh``.

All parameters are widened to float64 before the C code sees them (float32
and float16 values widen exactly), so finite differences can perturb them in
FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

# scale of the FP32 ambiguity band of every decision (1 = the error model of
# hm_oracle.c: or_mesh_raster's depth band and or_blend_errscale's bounds)
DEFAULT_BAND = 1.0


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_sort_order.restype = ctypes.c_int
        _lib.or_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(lib().or_num_threads())


def cam_array(cam) -> np.ndarray:
    """16 doubles: R (row-major), t, fx, fy, cx, cy."""
    if hasattr(cam, "as_array"):
        return _d(cam.as_array())
    return _d(np.concatenate([np.asarray(cam.R).reshape(9), np.asarray(cam.t).reshape(3),
                              [cam.fx, cam.fy, cam.cx, cam.cy]]))


def _pix(pix, W, H):
    if pix is None:
        return None, W * H
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    return pix, len(pix)


# --------------------------------------------------------------------------
# mesh
# --------------------------------------------------------------------------

def texture_unit(tex) -> np.ndarray:
    """Texture as float64 in [0,1]: RGB8 / 255, float textures as given."""
    t = np.asarray(tex)
    if t.dtype == np.uint8:
        return np.ascontiguousarray(t.astype(np.float64) / 255.0)
    return _d(t)


def mesh_raster(cam, mesh, bg=(0, 0, 0), znear=0.01, pix=None, tex=None):
    W, H = int(cam.width), int(cam.height)
    c = cam_array(cam)
    verts, uvs = _d(mesh.verts), _d(mesh.uvs)
    faces = np.ascontiguousarray(np.asarray(mesh.faces, dtype=np.int32))
    tx = texture_unit(mesh.texture) if tex is None else _d(tex)
    th, tw = tx.shape[:2]
    pix, n = _pix(pix, W, H)
    tri = np.empty(n, np.int32)
    dep = np.empty(n, np.float32)
    rgb = np.empty((3, n))
    uv = np.empty((2, n))
    bary = np.empty((3, n))
    d64 = np.empty(n)
    tol = np.empty(n)
    tri2 = np.empty(n, np.int32)
    tmg = np.empty(n)
    lib().or_mesh_raster(_p(c), W, H, _p(verts), _p(uvs), len(verts), _p(faces), len(faces),
                         _p(tx), tw, th, _p(_d(bg)), ctypes.c_double(znear),
                         _p(pix) if pix is not None else None, ctypes.c_int64(n),
                         _p(tri), _p(dep), _p(rgb), _p(uv), _p(bary), _p(d64), _p(tol), _p(tri2),
                         _p(tmg))
    return SimpleNamespace(tri_id=tri, depth=dep, rgb=rgb, uv=uv, bary=bary, depth64=d64,
                           depth_tol=tol, tri2=tri2, tri_margin=tmg)


def empty_mesh_result(n, bg=(0, 0, 0)):
    return SimpleNamespace(tri_id=np.full(n, -1, np.int32), depth=np.full(n, np.inf, np.float32),
                           rgb=np.repeat(_d(bg)[:, None], n, 1), uv=np.zeros((2, n)),
                           bary=np.zeros((3, n)), depth64=np.full(n, np.inf), depth_tol=np.zeros(n),
                           tri2=np.full(n, -1, np.int32), tri_margin=np.full(n, np.inf))


def mesh_raycast(cam, mesh, znear=0.01, pix=None):
    W, H = int(cam.width), int(cam.height)
    c = cam_array(cam)
    verts = _d(mesh.verts)
    faces = np.ascontiguousarray(np.asarray(mesh.faces, dtype=np.int32))
    pix, n = _pix(pix, W, H)
    tri = np.empty(n, np.int32)
    tz = np.empty(n)
    ed = np.empty(n)
    lib().or_mesh_raycast(_p(c), W, H, _p(verts), _p(faces), len(faces), ctypes.c_double(znear),
                          _p(pix) if pix is not None else None, ctypes.c_int64(n),
                          _p(tri), _p(tz), _p(ed))
    return SimpleNamespace(tri_id=tri, z=tz, edge_bary=ed)


# --------------------------------------------------------------------------
# Gaussians
# --------------------------------------------------------------------------

def sh_basis(deg: int, d) -> np.ndarray:
    d = _d(d)
    out = np.empty((deg + 1) ** 2)
    lib().or_sh_basis(deg, _p(d), _p(out))
    return out


def project(cam, g, W=None, H=None, filt3d=None, kernel2d=0.3, antialias=False):
    """Projection of every Gaussian for one camera; ``filt3d`` (per-Gaussian
    3D filter variance), ``kernel2d`` and ``antialias`` select the
    Mip-Splatting filters (``opac_scale`` is the opacity factor they imply)."""
    W = int(cam.width) if W is None else W
    H = int(cam.height) if H is None else H
    n = int(np.asarray(g.means).shape[0])
    c = cam_array(cam)
    means, scales, quats = _d(g.means), _d(g.scales), _d(g.quats)
    sh = _d(np.asarray(g.sh).astype(np.float64))
    f3 = _d(filt3d) if filt3d is not None else None
    vis = np.empty(n, np.int32)
    dep = np.empty(n, np.float32)
    m2 = np.empty((n, 2))
    cov = np.empty((n, 3))
    con = np.empty((n, 3))
    col = np.empty((n, 3))
    clamped = np.empty((n, 3), np.int32)
    osc = np.empty(n)
    op = _d(g.opacity) if getattr(g, "opacity", None) is not None else None
    lib().or_project(_p(c), W, H, n, _p(means), _p(scales), _p(quats), _p(op) if op is not None else None, _p(sh), int(g.sh_degree),
                     _p(f3) if f3 is not None else None, ctypes.c_double(kernel2d), int(bool(antialias)),
                     _p(vis), _p(dep), _p(m2), _p(cov), _p(con), _p(col), _p(clamped), _p(osc))
    return SimpleNamespace(visible=vis, depth=dep, mean2d=m2, cov2d=cov, conic=con, color=col,
                           clamped=clamped, opac_scale=osc)


def filter_3d(cameras, means, s2=0.2, near=0.2):
    """Mip-Splatting's 3D smoothing-filter variance per Gaussian (Yu et al.,
    CVPR 2024): v = s2 / nu^2 with nu the largest sampling rate f / z over
    the cameras that see the Gaussian's centre, f = max(fx, fy), z its view
    depth.  Readings: a camera sees the centre iff z > near and the
    projected centre lies in [0, W] x [0, H]; a Gaussian no camera sees gets
    v = 0 (no filter).  Plain FP64 numpy."""
    m = np.asarray(means, np.float64)
    best = np.zeros(len(m))                   # largest f / z so far (0: unseen)
    for cam in cameras:
        c = cam_array(cam)
        R, t = c[:9].reshape(3, 3), c[9:12]
        fx, fy, cx, cy = c[12:16]
        p = m @ R.T + t
        z = p[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = fx * p[:, 0] / z + cx
            w = fy * p[:, 1] / z + cy
            rate = max(fx, fy) / z
        seen = (z > near) & (u >= 0) & (u <= cam.width) & (w >= 0) & (w <= cam.height)
        best = np.where(seen & (rate > best), rate, best)
    with np.errstate(divide="ignore"):
        return np.where(best > 0, s2 / (best * best), 0.0)


def sort_order(proj) -> np.ndarray:
    n = len(proj.visible)
    order = np.empty(max(n, 1), np.int32)
    m = lib().or_sort_order(n, _p(proj.visible), _p(proj.depth), _p(order))
    return order[:m].copy()


# --------------------------------------------------------------------------
# blending
# --------------------------------------------------------------------------

def errscale(cam, proj) -> np.ndarray:
    """Per Gaussian (dm_x, dm_y, kappa_c): the scales of the FP32 error model
    of the blend's decisions (hm_oracle.c, or_blend_errscale)."""
    n = len(proj.visible)
    err = np.empty((max(n, 1), 3))
    lib().or_blend_errscale(_p(cam_array(cam)), n, _p(np.ascontiguousarray(proj.visible, np.int32)),
                            _p(_d(proj.mean2d)), _p(_d(proj.cov2d)), _p(err))
    return err


def _mesh_args(mesh_res):
    return (_p(np.ascontiguousarray(mesh_res.tri_id, dtype=np.int32)),
            _p(np.ascontiguousarray(mesh_res.depth, dtype=np.float32)),
            _p(_d(mesh_res.depth64)), _p(_d(mesh_res.depth_tol)), _p(_d(mesh_res.rgb)))


def _finish(out, mesh_res):
    """Per pixel `amb`: some decision of the walk, or the nearest-face
    decision of the mesh pass, lies inside its FP32 band."""
    out.amb = (out.n_amb > 0) | (np.asarray(mesh_res.tri_margin) < 1.0)
    return out


def blend(cam, proj, opacity, mesh_res, bg=(0, 0, 0), band=DEFAULT_BAND, pix=None, order=None):
    W, H = int(cam.width), int(cam.height)
    if order is None:
        order = sort_order(proj)
    order = np.ascontiguousarray(order, dtype=np.int32)
    pix, n = _pix(pix, W, H)
    err = errscale(cam, proj)
    rgb = np.empty((3, n))
    T = np.empty(n)
    nc = np.empty(n, np.int32)
    na = np.empty(n, np.int32)
    mg = np.empty(n)
    ev = np.empty(n, np.int64)
    fp = np.empty(n, np.uint64)
    lib().or_blend(W, H, len(proj.visible), _p(order), len(order), _p(proj.depth),
                   _p(_d(proj.mean2d)), _p(_d(proj.conic)), _p(_d(opacity)), _p(_d(proj.color)),
                   _p(err), *_mesh_args(mesh_res), _p(_d(bg)), ctypes.c_double(band),
                   _p(pix) if pix is not None else None, ctypes.c_int64(n),
                   _p(rgb), _p(T), _p(nc), _p(na), _p(mg), _p(ev), _p(fp))
    return _finish(SimpleNamespace(rgb=rgb, T=T, n_contrib=nc, n_amb=na, margin=mg, evaluated=ev,
                                   fp=fp), mesh_res)


def blend_grid(cam, proj, opacity, mesh_res, bg=(0, 0, 0), band=DEFAULT_BAND, cell=16, rows=None,
               order=None):
    """Full-image blend with the exact cell prefilter; ``rows=(r0, r1)``
    restricts the work to a band of rows (outputs elsewhere are undefined)."""
    W, H = int(cam.width), int(cam.height)
    if order is None:
        order = sort_order(proj)
    order = np.ascontiguousarray(order, dtype=np.int32)
    r0, r1 = (0, H) if rows is None else rows
    n = W * H
    err = errscale(cam, proj)
    rgb = np.zeros((3, n))
    T = np.zeros(n)
    nc = np.zeros(n, np.int32)
    na = np.zeros(n, np.int32)
    mg = np.zeros(n)
    ev = np.zeros(n, np.int64)
    fp = np.zeros(n, np.uint64)
    lib().or_blend_grid(W, H, cell, _p(order), len(order), _p(proj.depth), _p(_d(proj.mean2d)),
                        _p(_d(proj.cov2d)), _p(_d(proj.conic)), _p(_d(opacity)), _p(_d(proj.color)),
                        _p(err), *_mesh_args(mesh_res), _p(_d(bg)), ctypes.c_double(band),
                        int(r0), int(r1), _p(rgb), _p(T), _p(nc), _p(na), _p(mg), _p(ev), _p(fp))
    return _finish(SimpleNamespace(rgb=rgb, T=T, n_contrib=nc, n_amb=na, margin=mg, evaluated=ev,
                                   fp=fp), mesh_res)


def flip_outcomes(cam, proj, opacity, mesh_res, q, lin, bg=(0, 0, 0), band=DEFAULT_BAND,
                  order=None, err=None, max_flips=10):
    """Every outcome (rgb[3], T, n_contrib) of pixel `lin` (= y*W + x) that an
    FP32 renderer may validly produce: the walk re-run with each subset of
    its ambiguous decisions inverted (later decisions follow the flipped
    path).  `q` indexes the pixel in `mesh_res`.  Returns a list of
    (rgb, T, n) tuples, the unflipped walk first."""
    W = int(cam.width)
    x, y = int(lin % W), int(lin // W)
    if order is None:
        order = sort_order(proj)
    # the Gaussians whose inflated 3-sigma box holds the centre (the walk's
    # result only depends on those), in the global order
    m2, cov = np.asarray(proj.mean2d), np.asarray(proj.cov2d)
    o = np.asarray(order)
    hx = 3.0 * np.sqrt(1.01 * np.maximum(cov[o, 0], 0)) + 1.0
    hy = 3.0 * np.sqrt(1.01 * np.maximum(cov[o, 2], 0)) + 1.0
    near = (np.abs(x + 0.5 - m2[o, 0]) <= hx) & (np.abs(y + 0.5 - m2[o, 1]) <= hy)
    lst = np.ascontiguousarray(o[near], dtype=np.int32)
    err = errscale(cam, proj) if err is None else err
    hit = int(mesh_res.tri_id[q] >= 0)
    Im = _d(np.asarray(mesh_res.rgb)[:, q] if hit else bg)
    args = (_p(lst), len(lst), _p(proj.depth), _p(_d(proj.mean2d)), _p(_d(proj.conic)),
            _p(_d(opacity)), _p(_d(proj.color)), _p(err), hit,
            ctypes.c_float(float(mesh_res.depth[q])), ctypes.c_double(float(mesh_res.depth64[q])),
            ctypes.c_double(float(mesh_res.depth_tol[q])), _p(Im), ctypes.c_double(band))
    outs, seen, masks = [], {0}, [0]
    while masks:
        mask = masks.pop(0)
        rgb = np.empty(3)
        T = np.empty(1)
        nc = np.empty(1, np.int32)
        na = np.empty(1, np.int32)
        lib().or_blend_flipped(x, y, *args, ctypes.c_uint32(mask), _p(rgb), _p(T), _p(nc), _p(na))
        outs.append((rgb, float(T[0]), int(nc[0])))
        k = min(int(na[0]), max_flips)
        # masks over the ambiguous decisions this path meets, beyond what is queued
        for j in range(k):
            nm = mask | (1 << j)
            if nm not in seen:
                seen.add(nm)
                masks.append(nm)
    return outs


def render(scene, view=0, pix=None, band=DEFAULT_BAND, mode="brute", gaussians=None, tex=None,
           rows=None, znear=0.01, filt3d=None, kernel2d=0.3, antialias=False):
    """Full hybrid render of one view: mesh pass, projection, blend.  Returns
    a namespace with the mesh pass (``mesh``), the projection (``proj``) and
    the blend (``out``).  ``filt3d``, ``kernel2d``, ``antialias``: the
    Mip-Splatting filters (see ``project``)."""
    cam = scene.cameras[view]
    g = scene.gaussians if gaussians is None else gaussians
    bg = np.asarray(scene.bg, np.float64)
    W, H = int(cam.width), int(cam.height)
    if mode == "grid":
        pix = None
    n = W * H if pix is None else len(pix)
    if scene.mesh is not None:
        mr = mesh_raster(cam, scene.mesh, bg=bg, znear=znear, pix=pix, tex=tex)
    else:
        mr = empty_mesh_result(n, bg)
    pr = project(cam, g, filt3d=filt3d, kernel2d=kernel2d, antialias=antialias)
    opac = np.asarray(g.opacity, np.float64) * pr.opac_scale
    order = sort_order(pr)
    if mode == "grid":
        out = blend_grid(cam, pr, opac, mr, bg=bg, band=band, rows=rows, order=order)
    else:
        out = blend(cam, pr, opac, mr, bg=bg, band=band, pix=pix, order=order)
    return SimpleNamespace(mesh=mr, proj=pr, out=out, opacity=opac, cam=cam, bg=bg, pix=pix,
                           order=order, band=band)


def outcomes_at(orc, j):
    """flip_outcomes for entry j of a render() result (pixel pix[j], or j
    for a full image)."""
    lin = int(orc.pix[j]) if orc.pix is not None else int(j)
    if not hasattr(orc, "err"):
        orc.err = errscale(orc.cam, orc.proj)
    return flip_outcomes(orc.cam, orc.proj, orc.opacity, orc.mesh, j, lin, bg=orc.bg, band=orc.band,
                         order=orc.order, err=orc.err)
