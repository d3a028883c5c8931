"""hm_blend_backward_noalloc: the backward pass for callers that cannot
allocate device memory (code inside a stream capture, a plug-in whose host
owns the allocator, a real-time loop), with its scratch in the library's
static device array.  Its gradients must equal those of hm_blend_backward
with a caller workspace, on two calls in a row (the array keeps the previous
call's contents, so the second call checks that the entry point clears what
it needs).  The file sorts last so a run that stops at the first failure
has run every other test already; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2506_06988_b300 import lib, scenes
from paper_2506_06988_b300.render import MeshInput, Renderer

pytestmark = pytest.mark.gpu


def _scene():
    s = scenes.config0_scene(seed=3)
    s.mesh.texture = s.mesh.texture.astype(np.float32) / 255.0
    s.bg = np.array([0.1, 0.2, 0.3], np.float32)
    return s


def _grads_noalloc(r, P, mesh, dI, dT):
    th, tw = mesh.texture.shape[:2]
    g = r.grad_buffers((th, tw))
    r.opt.bwd_stages = 0
    st = lib.hm_blend_backward_noalloc(
        r.cams, r.n, P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], r.sh_degree,
        r.sh_format, r.records, r.pair_vals, r.ranges, r.mesh_depth, r.mesh_rgb, r.uv, tw, th,
        r.opt, r.T, r.last_idx, dI, dT, g["means"], g["scales"], g["quats"], g["opacity"], g["sh"],
        g["texture"], r.status_word, torch.cuda.current_stream().cuda_stream)
    lib.check(st, "hm_blend_backward_noalloc")
    return g


def test_noalloc_backward_matches_workspace_backward_twice():
    s = _scene()
    g = s.gaussians
    dev = "cuda"
    P = {k: torch.as_tensor(getattr(g, k), device=dev).contiguous() for k in ("means", "scales", "quats", "opacity", "sh")}
    mesh = MeshInput.from_numpy(s.mesh, device=dev)
    r = Renderer(s.cameras, g.n, g.sh_degree, n_verts=len(s.mesh.verts), n_faces=len(s.mesh.faces),
                 tex_shape=s.mesh.texture.shape, bg=tuple(s.bg), device=dev)
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    dI = torch.randn(3 * r.npix, device=dev, generator=gen)
    dT = torch.randn(r.npix, device=dev, generator=gen)
    ref = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], dI, dT, mesh=mesh,
                     tex_grad=True)
    for _ in range(2):
        got = _grads_noalloc(r, P, mesh, dI, dT)
        torch.cuda.synchronize()
        for k, v in ref.items():
            # same kernels; only the order of FP32 atomic additions may differ
            tol = 1e-5 * float(v.abs().max()) + 1e-12
            assert torch.allclose(got[k], v, rtol=1e-5, atol=tol), k


def test_noalloc_rejects_problems_above_its_static_scratch():
    cams = lib.cameras([scenes._identity_cam(16, 16)])
    o = lib.options()
    n_max = (lib.HM_BWD_NOALLOC_BYTES - 256) // (9 * 4)
    st = lib.hm_blend_backward_noalloc(cams, n_max + 1, 16, 16, 16, 16, 16, 0, lib.HM_SH_F32, 16, 16,
                                       16, None, None, None, 0, 0, o, 16, 16, 16, None, 16, 16, 16, 16,
                                       16, None, None, 0)
    assert st == lib.HM_ERR_INVALID_ARG
    assert "static array" in lib.last_error()
