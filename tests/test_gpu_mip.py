"""The Mip-Splatting back-end (Tab. 1 pairs the mesh with it; filters as
published by Yu et al., CVPR 2024) on the GPU against the oracle: the 3D
smoothing variance (hm_mip_filter_3d), the projection with the 3D filter
and the 2D Mip filter (records), the hybrid render and its gradients.

The 3D variance fed to the projection comes from the oracle (rounded to
FP32, widened again for the oracle), so both sides filter with the same
numbers.  Tolerances as for the 3DGS kernel: conics 1e-4 of their scale,
images 1e-4 outside the FP32/FP64 ambiguity band, gradients 1e-3; the
opacity factors are FP32 products and square roots (relative 1e-5)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import torch_ref as TR
from paper_2506_06988_b300 import scenes

from gpu_util import check_grad, compare_blend, gaussians_to_torch, make_renderer, records_np, view_outputs  # noqa: E402,E501

pytestmark = pytest.mark.gpu


def _room(seed=21, res=((160, 120), (200, 90), (128, 128)), n_gauss=4000):
    return scenes.room_scene(seed, n_tris=3000, n_gauss=n_gauss, resolutions=res,
                             focal_per_width=1100.0 / 1920.0)


def _f3(scene, s2=0.2):
    v = O.filter_3d(scene.cameras, scene.gaussians.means, s2=s2).astype(np.float32)
    return v, v.astype(np.float64)


def _mip_render(scene, v32, **kw):
    r = make_renderer(scene, mip=True, **kw)
    r.set_filter_3d(torch.as_tensor(v32, device="cuda"))
    P = gaussians_to_torch(scene.gaussians)
    from paper_2506_06988_b300.render import MeshInput
    mesh = MeshInput.from_numpy(scene.mesh) if scene.mesh is not None else None
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)
    torch.cuda.synchronize()
    return r, P, mesh


def test_filter_3d_kernel_matches_oracle():
    s = _room()
    m = np.asarray(s.gaussians.means, np.float64)
    # Gaussians whose visibility decision is within reach of FP32 rounding in
    # some camera (centre within 1e-3 px of the image edge, depth within 1e-6
    # of the near plane) are left out of the comparison
    amb = np.zeros(len(m), bool)
    for cam in s.cameras:
        c = O.cam_array(cam)
        p = m @ c[:9].reshape(3, 3).T + c[9:12]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = c[12] * p[:, 0] / p[:, 2] + c[14]
            w = c[13] * p[:, 1] / p[:, 2] + c[15]
        near_edge = (np.minimum.reduce([np.abs(u), np.abs(u - cam.width), np.abs(w), np.abs(w - cam.height)]) < 1e-3)
        amb |= (p[:, 2] > 0.2) & near_edge | (np.abs(p[:, 2] - 0.2) < 1e-6)
    want = O.filter_3d(s.cameras, m, s2=0.2)
    r = make_renderer(s, mip=True)
    got = r.mip_filter_3d(torch.as_tensor(np.asarray(s.gaussians.means, np.float32), device="cuda"), s2=0.2)
    got = got.cpu().numpy().astype(np.float64)
    ok = ~amb
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok] > 0, want[ok] > 0)
    assert np.all(np.abs(got[ok] - want[ok]) <= 2e-6 * want[ok] + 1e-30)
    assert (want > 0).sum() > 300                        # room cameras see a fifth of the Gaussians


def test_mip_records_match_oracle():
    s = _room(res=((160, 120), (200, 90)))
    v32, v64 = _f3(s)
    r, _, _ = _mip_render(s, v32)
    rec = records_np(r)
    n = s.gaussians.n
    for k, cam in enumerate(s.cameras):
        p = O.project(cam, s.gaussians, filt3d=v64, kernel2d=0.1, antialias=True)
        sl = slice(k * n, (k + 1) * n)
        assert np.array_equal(rec.depth[sl], p.depth)
        on = p.visible.astype(bool) & (rec.x0[sl] <= rec.x1[sl])
        scale = np.sqrt(np.abs(p.conic[on, 0] * p.conic[on, 2]))
        c_err = np.abs(rec.conic[sl][on] - p.conic[on]) / scale[:, None]
        assert c_err.max() < 1e-4, c_err.max()
        want_op = np.asarray(s.gaussians.opacity, np.float64)[on] * p.opac_scale[on]
        assert np.all(np.abs(rec.opacity[sl][on] - want_op) <= 1e-5 * want_op + 1e-9)
        assert (p.opac_scale[on] < 1).mean() > 0.9           # the filters do act


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_mip_hybrid_render_config0(tile):
    s = scenes.config0_scene(seed=5)
    v32, v64 = _f3(s)
    r, _, _ = _mip_render(s, v32, tile=tile)
    orc = O.render(s, 0, filt3d=v64, kernel2d=0.1, antialias=True)
    st = compare_blend(view_outputs(r, 0), orc)
    assert st["amb_frac"] < 2e-3, st


def test_mip_backward_matches_gradient_oracle():
    s = scenes.config0_scene(seed=6)
    s.bg = np.array([0.2, 0.3, 0.4], np.float32)
    v32, v64 = _f3(s)
    flt = dict(filt3d=v64, kernel2d=0.1, antialias=True)
    npx = s.cameras[0].n_pixels
    rng = np.random.default_rng(2)
    gI = rng.standard_normal((3, npx))
    gT = rng.standard_normal(npx)
    orc = O.render(s, **flt)
    amb = orc.out.amb
    gI[:, amb] = 0.0
    gT[amb] = 0.0
    _, ref = TR.render_grad(s, 0, gI, gT, tex=O.texture_unit(s.mesh.texture), **flt)
    r, P, mesh = _mip_render(s, v32)
    g = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"],
                   torch.as_tensor(gI.reshape(-1), dtype=torch.float32, device="cuda"),
                   torch.as_tensor(gT, dtype=torch.float32, device="cuda"), mesh=mesh, tex_grad=True)
    torch.cuda.synchronize()
    for k in ("means", "scales", "quats", "opacity", "sh"):
        check_grad(k, g[k].cpu().numpy(), ref[k])
