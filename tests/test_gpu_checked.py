"""The index-checked library (libhm_checked.so, built with HM_CHECKED):
on valid inputs every check passes and the outputs equal the default
library's bit for bit; on a corrupt input that the default build would
follow out of the tile's list -- a stop position beyond the list's end --
the check reports HM_DEV_BAD_INDEX through hm_checked_status and the access
is skipped.  The corrupt input is given to the checked library only."""
import pytest
import torch

from paper_2506_06988_b300 import lib, scenes
from paper_2506_06988_b300.render import MeshInput, Renderer

from gpu_util import gaussians_to_torch

pytestmark = pytest.mark.gpu


def _frame(seed=21):
    s = scenes.room_scene(seed, n_tris=3000, n_gauss=5000, resolutions=((160, 120), (96, 64)),
                          focal_per_width=1100.0 / 1920.0)
    g = s.gaussians
    P = gaussians_to_torch(g)
    PM = (P["means"], P["scales"], P["quats"], P["opacity"], P["sh"])
    mesh = MeshInput.from_numpy(s.mesh, device="cuda")
    r = Renderer(s.cameras, g.n, g.sh_degree, n_verts=len(s.mesh.verts), n_faces=len(s.mesh.faces),
                 tex_shape=s.mesh.texture.shape, bg=tuple(s.bg), device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    dI = torch.randn(3 * r.npix, device="cuda", generator=gen)
    return r, PM, mesh, dI


def _run(r, PM, mesh, dI):
    r.render(*PM, mesh)
    g = r.backward(*PM, dI, None, mesh=mesh, tex_grad=True)
    torch.cuda.synchronize()
    out = {k: getattr(r, k).clone() for k in ("rgb", "T", "n_contrib", "last_idx", "tri_id", "mesh_depth",
                                              "pair_vals", "ranges")}
    out.update({"d_" + k: v.clone() for k, v in g.items()})
    return out


def test_checked_library_passes_valid_frames_and_matches():
    r, PM, mesh, dI = _frame()
    ref = _run(r, PM, mesh, dI)
    before = lib.use(lib.load_checked())
    try:
        assert lib.hm_checked_status(reset=True) in (0, lib.HM_DEV_BAD_INDEX)   # clear earlier state
        got = _run(r, PM, mesh, dI)
        assert lib.hm_checked_status(reset=True) == 0
        assert r.status()[0] == 0
    finally:
        lib.use(before)
    n = int(r.n_pairs.item())
    for k in ("rgb", "T", "n_contrib", "last_idx", "tri_id", "mesh_depth", "ranges"):
        assert torch.equal(got[k], ref[k]), k
    assert torch.equal(got["pair_vals"][:n], ref["pair_vals"][:n])
    for k in ("d_means", "d_scales", "d_quats", "d_opacity", "d_sh", "d_texture"):
        # the same kernels; only the order of FP32 atomic additions may differ
        tol = 1e-5 * float(ref[k].abs().max()) + 1e-12
        assert torch.allclose(got[k], ref[k], rtol=1e-5, atol=tol), k


@pytest.mark.plants_bad_index
def test_checked_library_reports_a_stop_position_beyond_the_list():
    r, PM, mesh, dI = _frame(seed=22)
    before = lib.use(lib.load_checked())
    try:
        lib.hm_checked_status(reset=True)
        r.render(*PM, mesh)
        torch.cuda.synchronize()
        assert lib.hm_checked_status(reset=True) == 0
        hit = torch.nonzero(r.last_idx > 0)
        assert hit.numel() > 0
        r.last_idx[int(hit[0])] = 0x7FFFFFFF            # beyond every list
        g = r.backward(*PM, dI, None, mesh=mesh, tex_grad=True)
        torch.cuda.synchronize()
        assert lib.hm_checked_status(reset=True) == lib.HM_DEV_BAD_INDEX
        assert all(bool(torch.isfinite(v).all()) for v in g.values())
    finally:
        lib.use(before)
