"""hm_mesh_prune (the mesh-pruning metrics of Sec. 3.3 / Algorithm 1 stage
1) against the pruning oracle: flags and piece labels bit for bit -- every
decision is defined in FP64 without fused operations (normals, areas, the
angle test) or in FP32 in a fixed order (the normal-map variation), and the
ranks are exact -- on the oracle pins' meshes and on a room mesh seen by
three cameras with seeded prior normal maps."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import prune as PO
from paper_2506_06988_b300 import lib, scenes

from test_oracle_prune import _hinge, grid  # noqa: E402

pytestmark = pytest.mark.gpu


def _gpu_prune(verts, faces, cams=None, tri_ids=None, normals=None, **kw):
    v = torch.as_tensor(np.asarray(verts, np.float32), device="cuda").contiguous()
    f = torch.as_tensor(np.asarray(faces, np.int32), device="cuda").contiguous()
    nv, nf = len(verts), len(faces)
    cam_arr = lib.cameras(cams) if cams else None
    tri = nrm = None
    if cams:
        tri = torch.as_tensor(np.concatenate([np.asarray(t, np.int32).reshape(-1) for t in tri_ids]), device="cuda")
        nrm = torch.as_tensor(np.concatenate([np.asarray(n, np.float32).reshape(-1) for n in normals]), device="cuda")
    p = lib.prune_params(**kw)
    ws = torch.empty(max(1, lib.hm_mesh_prune_workspace_size(cam_arr, nv, nf)), dtype=torch.uint8, device="cuda")
    flags = torch.empty(nf, dtype=torch.uint8, device="cuda")
    label = torch.empty(nf, dtype=torch.int32, device="cuda")
    lib.check(lib.hm_mesh_prune(cam_arr, v, nv, f, nf, tri, nrm, p, flags, label, ws, ws.numel(),
                                torch.cuda.current_stream().cuda_stream), "hm_mesh_prune")
    return flags.cpu().numpy(), label.cpu().numpy()


def _compare(verts, faces, cams=None, tri_ids=(), normals=(), **kw):
    gf, gl = _gpu_prune(verts, faces, cams, list(tri_ids), list(normals), **kw)
    of, _, ol = PO.prune(verts, faces, list(tri_ids), list(normals), **kw)
    assert np.array_equal(gf, of), (np.nonzero(gf != of)[0][:10], gf[gf != of][:10], of[gf != of][:10])
    assert np.array_equal(gl, ol)
    return gf


@pytest.mark.parametrize("deg", [30.0, 60.0])
def test_prune_hinge(deg):
    v, f = _hinge(deg)
    _compare(v, f, alpha_area=0.0, alpha_group=1)


def test_prune_grids_and_pieces():
    v1, f1 = grid(5, 5)
    v2, f2 = grid(15, 5, x0=100.0)
    v = np.concatenate([v1, v2])
    f = np.concatenate([f1, f2 + len(v1)])
    fl = _compare(v, f, alpha_area=10.0, alpha_group=100)
    assert (fl & PO.F_GROUP).any() and (fl & PO.F_AREA).any()


def test_prune_room_with_normal_maps():
    s = scenes.room_scene(13, n_tris=4000, n_gauss=100, resolutions=((160, 120), (200, 90), (96, 96)),
                          focal_per_width=1100.0 / 1920.0)
    tri = [O.mesh_raster(c, s.mesh, bg=s.bg).tri_id for c in s.cameras]
    nm = scenes.prior_normal_maps(s.cameras, seed=3)
    # weld coincident vertices so that walls share their corner edges (90 degrees)
    uniq, inv = np.unique(np.asarray(s.mesh.verts, np.float32), axis=0, return_inverse=True)
    s.mesh.verts, s.mesh.faces = uniq, inv.reshape(-1)[s.mesh.faces]
    for kw in (dict(), dict(alpha_normal=5.0, alpha_area=20.0, angle_deg=30.0, alpha_group=10)):
        fl = _compare(s.mesh.verts, s.mesh.faces, s.cameras, tri, nm, **kw)
        for bit in (PO.F_NORMAL, PO.F_ANGLE, PO.F_AREA):
            assert (fl & bit).any(), (bit, kw)


def test_prune_rejects_bad_face_indices():
    v, f = grid(2, 2)
    f = f.copy()
    f[3, 1] = 999
    with pytest.raises(lib.HmError, match="out of range"):
        _gpu_prune(v, f)
