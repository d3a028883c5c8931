"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs, and compare them.

Tolerances (derived in the design notes):
* mesh tri_id, Gaussian depth keys, sorted pair lists, tile ranges and
  per-pixel Gaussian counts are compared bit-exactly; the mesh depth within
  the FP32 band the oracle states per pixel (a few ulps of the FP64 depth);
* images and T within 1e-4 absolute per channel;
* threshold decisions (3-sigma cut, alpha >= 1/255, T >= 1e-4, the mesh cut,
  the nearest face) are taken in FP32 on the GPU and FP64 in the oracle; the
  oracle states per decision the band an FP32 evaluation can move it by.  A
  pixel with a decision inside its band is "ambiguous": its GPU result must
  equal (count exactly, colour and T within 1e-4) one of the outcomes the
  oracle lists by re-walking the pixel with each subset of those decisions
  inverted.  Every other pixel is compared directly.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np
import torch

from oracle import oracle as O
from paper_2506_06988_b300 import lib
from paper_2506_06988_b300.render import MeshInput, Renderer

IMG_TOL = 1e-4


def check_grad(name, g, ref, rel=1e-3, floor=1e-4):
    """GPU gradient vs the FP64 oracle: ||g - ref|| <= rel ||ref|| and per
    element |g - ref| <= rel |ref| + floor max|ref| (the floor absorbs FP32
    atomic accumulation order on near-cancelling sums)."""
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nref = np.linalg.norm(ref)
    assert nref > 0, name
    norm_err = np.linalg.norm(g - ref) / nref
    el = np.abs(g - ref) <= rel * np.abs(ref) + floor * np.abs(ref).max()
    assert norm_err <= rel, (name, norm_err)
    assert el.all(), (name, int((~el).sum()), float(np.abs(g - ref).max()))
    return norm_err


def gaussians_to_torch(g, device="cuda"):
    t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), device=device).to(dt)  # noqa: E731
    sh = torch.as_tensor(np.ascontiguousarray(g.sh), device=device)
    return dict(means=t(g.means), scales=t(g.scales), quats=t(g.quats), opacity=t(g.opacity), sh=sh)


def make_renderer(scene, tile=(16, 16), batch=None, mesh_cull=True, views=None, **kw):
    cams = scene.cameras if views is None else [scene.cameras[v] for v in views]
    g = scene.gaussians
    m = scene.mesh
    return Renderer(cams, g.n, g.sh_degree, sh_f16=(np.asarray(g.sh).dtype == np.float16),
                    n_verts=0 if m is None else len(m.verts), n_faces=0 if m is None else len(m.faces),
                    tex_shape=None if m is None else m.texture.shape, tile=tile, batch=batch,
                    mesh_cull=mesh_cull, bg=tuple(np.asarray(scene.bg, np.float64)), **kw)


def gpu_render(scene, tile=(16, 16), batch=None, mesh_cull=True, views=None, **kw):
    r = make_renderer(scene, tile, batch, mesh_cull, views, **kw)
    P = gaussians_to_torch(scene.gaussians)
    mesh = MeshInput.from_numpy(scene.mesh) if scene.mesh is not None else None
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)
    torch.cuda.synchronize()
    return r, P, mesh


def view_outputs(r: Renderer, k: int):
    """numpy outputs of camera k (flat per pixel; rgb planar [3, npix])."""
    w, h = r.sizes[k]
    a, b = int(r.pix_off[k]), int(r.pix_off[k + 1])
    out = SimpleNamespace(
        rgb=r.rgb[3 * a:3 * b].view(3, -1).cpu().numpy().astype(np.float64),
        T=r.T[a:b].cpu().numpy().astype(np.float64),
        n_contrib=r.n_contrib[a:b].cpu().numpy(),
        last_idx=r.last_idx[a:b].cpu().numpy())
    if r.has_mesh:
        out.tri_id = r.tri_id[a:b].cpu().numpy()
        out.depth = r.mesh_depth[a:b].cpu().numpy()
        out.mesh_rgb = r.mesh_rgb[3 * a:3 * b].view(3, -1).cpu().numpy().astype(np.float64)
        out.uv = r.uv[2 * a:2 * b].view(2, -1).cpu().numpy().astype(np.float64)
    return out


def compare_mesh(gout, m, pix=None, rgb_tol=1e-4, uv_tol=1e-6):
    """GPU mesh pass vs the oracle's (``O.mesh_raster`` over the same pixel
    list): tri_id bit-exact where the nearest-face decision is outside its
    FP32 band, else one of the two nearest covering faces; depth within the
    oracle's band of its FP64 depth; texel colour and UV close where the
    faces agree.  Returns statistics."""
    if pix is None:
        g_tri, g_dep, g_rgb, g_uv = gout.tri_id, gout.depth, gout.mesh_rgb, gout.uv
    else:
        g_tri, g_dep, g_rgb, g_uv = gout.tri_id[pix], gout.depth[pix], gout.mesh_rgb[:, pix], gout.uv[:, pix]
    amb = m.tri_margin < 1.0
    same = g_tri == m.tri_id
    assert same[~amb].all(), ("tri_id", int((~same & ~amb).sum()))
    assert np.array_equal(g_tri[~same], m.tri2[~same]), "tri_id: neither of the two nearest faces"
    hit = same & (m.tri_id >= 0)
    derr = np.abs(g_dep[hit].astype(np.float64) - m.depth64[hit])
    assert (derr <= m.depth_tol[hit]).all(), ("depth", float((derr / m.depth_tol[hit]).max()))
    assert np.all(np.isinf(g_dep[m.tri_id < 0]))
    assert np.abs(g_rgb[:, same] - m.rgb[:, same]).max(initial=0.0) <= rgb_tol
    assert np.abs(g_uv[:, same] - m.uv[:, same]).max(initial=0.0) <= uv_tol
    return dict(pixels=len(g_tri), tri_ambiguous=int(amb.sum()), tri_swapped=int((~same).sum()),
                depth_err_in_band=float((derr / m.depth_tol[hit]).max(initial=0.0)),
                depth_exact_fp32=float((g_dep[hit] == m.depth[hit]).mean()) if hit.any() else 1.0)


def compare_blend(gout, orc, pix=None, tol=IMG_TOL):
    """GPU image vs the oracle's render (``O.render`` of the same view and
    pixel list).  Unambiguous pixels: counts exact, colour and T within
    `tol`.  Ambiguous pixels: the GPU result must be one of the valid
    outcomes (``O.outcomes_at``).  Returns statistics; raises
    AssertionError on a failure."""
    o = orc.out
    sel = slice(None) if pix is None else pix
    g_rgb, g_T, g_n = gout.rgb[:, sel], gout.T[sel], gout.n_contrib[sel]
    g_tri = gout.tri_id[sel] if hasattr(gout, "tri_id") else None
    amb = np.asarray(o.amb, bool)
    ok = ~amb
    d_rgb = np.abs(g_rgb - o.rgb).max(0)
    d_T = np.abs(g_T - o.T)
    n_bad = int((g_n[ok] != o.n_contrib[ok]).sum())
    stats = dict(pixels=len(g_T), ambiguous=int(amb.sum()), amb_frac=float(amb.mean()),
                 max_rgb_err=float(d_rgb[ok].max()) if ok.any() else 0.0,
                 max_T_err=float(d_T[ok].max()) if ok.any() else 0.0,
                 count_mismatch=n_bad)
    if n_bad:
        bad = np.nonzero(ok & (g_n != o.n_contrib))[0]
        stats["bad_margins"] = o.margin[bad][:10].tolist()
    assert n_bad == 0, stats
    assert stats["max_rgb_err"] <= tol, stats
    assert stats["max_T_err"] <= tol, stats
    # ambiguous pixels: the GPU took one of the valid paths
    flipped = swapped = 0
    for j in np.nonzero(amb)[0]:
        if g_tri is not None and g_tri[j] != orc.mesh.tri_id[j]:
            swapped += 1          # the other face of an ambiguous nearest-face decision (compare_mesh)
            assert orc.mesh.tri_margin[j] < 1.0 and g_tri[j] == orc.mesh.tri2[j], (j, stats)
            continue
        outs = O.outcomes_at(orc, j)
        match = [k for k, (rgb, T, n) in enumerate(outs)
                 if n == g_n[j] and np.abs(rgb - g_rgb[:, j]).max() <= tol and abs(T - g_T[j]) <= tol]
        assert match, (j, "no valid outcome", [(n, T) for _, T, n in outs], int(g_n[j]), float(g_T[j]))
        flipped += int(match[0] != 0)
    stats.update(amb_took_flipped=flipped, amb_other_face=swapped)
    return stats


def oracle_view(scene, view, pix=None, mode="brute"):
    return O.render(scene, view, pix=pix, mode=mode)


# the records hold the conic pre-multiplied by K = -log2(e)/2 (xy by 2K)
K_CONIC = np.float64(np.float32(-0.72134752044448170))


def records_np(r: Renderer):
    rec = r.records_view().cpu().numpy()
    u32 = rec.view(np.uint32)
    conic = rec[:, [2, 3, 4]].astype(np.float64) / np.array([K_CONIC, 2 * K_CONIC, K_CONIC])
    return SimpleNamespace(mean=rec[:, 0:2].astype(np.float64), conic=conic,
                           opacity=rec[:, 5], depth=rec[:, 6], color=rec[:, 8:11].astype(np.float64),
                           x0=u32[:, 7] & 0xFFFF, x1=u32[:, 7] >> 16, y0=u32[:, 11] & 0xFFFF,
                           y1=u32[:, 11] >> 16)


def expected_pairs(r: Renderer, rec, tile_max=None):
    """Per global tile, the record indices a correct bin/sort must list:
    records whose tile range covers the tile (and, with the cull, whose depth
    is below the tile's farthest mesh depth), ordered by (depth, index)."""
    V, n = r.V, r.n
    lists = [[] for _ in range(r.ntiles)]
    tw, th = r.opt.tile_w, r.opt.tile_h
    tile_off = 0
    for v in range(V):
        w, h = r.sizes[v]
        tx_n = (w + tw - 1) // tw
        ty_n = (h + th - 1) // th
        for i in range(n):
            it = v * n + i
            x0, x1, y0, y1 = int(rec.x0[it]), int(rec.x1[it]), int(rec.y0[it]), int(rec.y1[it])
            if x0 > x1 or y0 > y1:
                continue
            for ty in range(y0, y1 + 1):
                for tx in range(x0, x1 + 1):
                    gt = tile_off + ty * tx_n + tx
                    if tile_max is not None and not (rec.depth[it] < tile_max[gt]):
                        continue
                    lists[gt].append(it)
        tile_off += tx_n * ty_n
    for gt in range(r.ntiles):
        lists[gt].sort(key=lambda it: (rec.depth[it], it))
    return lists
