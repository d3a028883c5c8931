"""Batched views of uneven resolution, CUDA-graph frames and the autotuner.

* A frame captured in a CUDA graph (GraphStep) gives exactly the eager
  frame's images and counts, and its gradients up to the order of FP32
  atomic additions; a replay reads the parameters' current contents.
* The autotuner times every valid (tile, batch) pair; the image it leads to
  is bit-identical to the default configuration's (per-pixel candidate sets
  and their order do not depend on the tile or the staging batch).
* Gradients of a batched render of several cameras of different sizes with
  FP16 SH storage equal the sum over cameras of the FP64 gradient oracle.
* The chunked renderer (one chunk's lists at a time, recomputed in the
  backward pass) reproduces the batched renderer's images and gradients.
* The persistent launch (resident CTAs claiming (view, tile) work from a
  counter) gives the grid launch's images bit for bit, its gradients up to
  atomic order, and matches the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import torch_ref as TR
from paper_2506_06988_b300 import autotune, scenes
from paper_2506_06988_b300.render import GraphStep, MeshInput

from gpu_util import (check_grad, compare_blend, gaussians_to_torch, gpu_render, make_renderer,  # noqa: E402
                      oracle_view, view_outputs)

pytestmark = pytest.mark.gpu

RES = ((160, 120), (96, 64), (200, 104))


def _room(seed=31, res=RES, n_gauss=4000, n_tris=2500, sh_f16=True):
    return scenes.room_scene(seed, n_tris=n_tris, n_gauss=n_gauss, resolutions=res, sh_f16=sh_f16,
                             focal_per_width=1100.0 / 1920.0)


def _params(P):
    return (P["means"], P["scales"], P["quats"], P["opacity"], P["sh"])


def _grads_close(a, b):
    for k in b:
        tol = 1e-5 * float(b[k].abs().max()) + 1e-12
        assert torch.allclose(a[k], b[k], rtol=1e-5, atol=tol), k


def test_graph_step_matches_eager_frame():
    s = _room()
    r, P, mesh = gpu_render(s)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    dI = torch.randn(3 * r.npix, device="cuda", generator=gen)
    ref_g = r.backward(*_params(P), dI, None, mesh=mesh, tex_grad=True)
    # (last_idx is a position in the pair buffer: the graph bins without the
    # tile mesh cull, which shifts every tile's list; the gradients check it)
    ref = {k: getattr(r, k).clone() for k in ("rgb", "T", "n_contrib")}
    gs = GraphStep(r, _params(P), mesh, dL_drgb=dI, tex_grad=True)
    for _ in range(2):
        for k in ref:
            getattr(r, k).fill_(-1)
        gs.replay(check=True)
        torch.cuda.synchronize()
        for k, v in ref.items():
            assert torch.equal(getattr(r, k), v), k
        _grads_close(gs.grads, ref_g)


@pytest.mark.parametrize("lambda_ssim", [0.0, 0.2])
def test_graph_step_with_target_matches_eager_loss(lambda_ssim):
    # the graph decodes the uint8 target, evaluates the loss and back-propagates
    # it: the loss terms equal the eager hm_hybrid_loss on the decoded target,
    # and the gradients the eager backward of its dL/dI
    from paper_2506_06988_b300 import lib
    s = _room(seed=33)
    r, P, mesh = gpu_render(s)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    tgt8 = torch.randint(0, 256, (3 * r.npix,), dtype=torch.uint8, device="cuda", generator=gen)
    tgt = torch.from_numpy(tgt8.cpu().numpy().astype(np.float32) / np.float32(255.0)).cuda()
    lp = lib.loss_params(lambda_ssim=lambda_ssim, lambda_t=0.0)
    terms, dI, _ = r.loss(tgt, lp, texture_loss=False)
    ref_terms = terms.clone()
    ref_g = r.backward(*_params(P), dI.clone(), None, mesh=mesh, tex_grad=True)
    gs = GraphStep(r, _params(P), mesh, target=tgt8, loss_params=lp, tex_grad=True)
    gs.replay(check=True)
    torch.cuda.synchronize()
    assert torch.equal(gs.loss_terms, ref_terms)
    _grads_close(gs.grads, ref_g)


def test_graph_step_with_texture_loss_matches_eager():
    # a float32 target with the transmittance-aware texture loss on: the graph
    # passes dL/dI_m to the texel gradients like the eager call does
    from paper_2506_06988_b300 import lib
    s = _room(seed=34)
    r, P, mesh = gpu_render(s)
    mesh = MeshInput(mesh.verts, mesh.uvs, mesh.faces, mesh.texture.float() / 255.0
                     if mesh.texture.dtype == torch.uint8 else mesh.texture)
    r.render(*_params(P), mesh)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    tgt = torch.rand(3 * r.npix, device="cuda", generator=gen)
    lp = lib.loss_params(lambda_ssim=0.2, lambda_t=0.1)
    terms, dI, dM = r.loss(tgt, lp, texture_loss=True)
    assert dM is not None
    ref_terms = terms.clone()
    ref_g = r.backward(*_params(P), dI.clone(), None, mesh=mesh, tex_grad=True, dL_dmesh=dM.clone())
    gs = GraphStep(r, _params(P), mesh, target=tgt, loss_params=lp, tex_grad=True)
    gs.replay(check=True)
    torch.cuda.synchronize()
    assert torch.equal(gs.loss_terms, ref_terms)
    assert float(ref_terms[2]) > 0.0
    _grads_close(gs.grads, ref_g)


def test_decode_u8_is_exact():
    from paper_2506_06988_b300 import lib
    for n in (0, 5, 16, 1000, 4099):
        src = torch.arange(n, dtype=torch.int64).mul(37).remainder(256).to(torch.uint8).cuda()
        dst = torch.full((max(n, 1),), -1.0, device="cuda")
        lib.check(lib.hm_decode_u8(src, n, dst, torch.cuda.current_stream().cuda_stream), "hm_decode_u8")
        torch.cuda.synchronize()
        want = src.cpu().numpy().astype(np.float32) / np.float32(255.0)
        assert np.array_equal(dst[:n].cpu().numpy(), want)


@pytest.mark.parametrize("lam_ssim, lam_t", [(0.0, 0.0), (0.0, 0.1), (0.2, 0.1)])
def test_u8_target_loss_equals_the_decoded_target_loss(lam_ssim, lam_t):
    """hm_hybrid_loss_u8 reads each 8-bit code as code / 255 (correctly
    rounded): its loss terms and both gradients equal hm_hybrid_loss on the
    image hm_decode_u8 writes, bit for bit (pointwise L1 path and SSIM path
    with the texture loss)."""
    from paper_2506_06988_b300 import lib
    s = _room(seed=34, res=((160, 120), (96, 64)))
    r, P, mesh = gpu_render(s)
    r.render(*_params(P), mesh)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(6)
    codes = torch.randint(0, 256, (3 * r.npix,), device="cuda", generator=gen, dtype=torch.int32).to(torch.uint8)
    dec = torch.empty(3 * r.npix, device="cuda")
    lib.check(lib.hm_decode_u8(codes, codes.numel(), dec, torch.cuda.current_stream().cuda_stream), "hm_decode_u8")
    lp = lib.loss_params(lambda_ssim=lam_ssim, lambda_t=lam_t)
    t_f, dI_f, dM_f = (x.clone() if x is not None else None for x in r.loss(dec, lp, texture_loss=lam_t > 0))
    t_u, dI_u, dM_u = r.loss(codes, lp, texture_loss=lam_t > 0)
    torch.cuda.synchronize()
    assert torch.equal(t_u, t_f)
    assert torch.equal(dI_u, dI_f)
    if lam_t > 0:
        assert torch.equal(dM_u, dM_f)


def test_graph_step_copies_its_loss_to_pinned_host_memory():
    """GraphStep(loss_host=...): the replay's last node writes the loss terms
    to the pinned host buffer -- equal to the device terms -- and a second
    replay against another target updates it."""
    from paper_2506_06988_b300 import lib
    s = _room(seed=35, res=((160, 120), (96, 64)))
    r, P, mesh = gpu_render(s)
    r.render(*_params(P), mesh)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(8)
    target = torch.randint(0, 256, (3 * r.npix,), device="cuda", generator=gen, dtype=torch.int32).to(torch.uint8)
    host = torch.zeros(4, dtype=torch.float64).pin_memory()
    lp = lib.loss_params(lambda_ssim=0.0, lambda_t=0.1)
    gs = GraphStep(r, _params(P), mesh, target=target, loss_params=lp, tex_grad=True, loss_host=host)
    gs.replay()
    torch.cuda.synchronize()
    assert torch.equal(host, gs.loss_terms.cpu()) and float(host[3]) > 0.0
    first = host.clone()
    target.copy_(255 - target)                    # in place: the graph reads the new target
    gs.replay()
    torch.cuda.synchronize()
    assert torch.equal(host, gs.loss_terms.cpu()) and not torch.equal(host, first)
    with pytest.raises(ValueError):
        GraphStep(r, _params(P), mesh, target=target, loss_params=lp, loss_host=torch.zeros(4, dtype=torch.float64))


def test_graph_step_reads_current_parameters():
    s = _room(seed=32)
    r, P, mesh = gpu_render(s)
    gs = GraphStep(r, _params(P), mesh)
    P["means"][::3] += 0.02                      # in place: the graph sees the new values
    P["opacity"].mul_(0.9)
    gs.replay(check=True)
    torch.cuda.synchronize()
    got = (r.rgb.clone(), r.T.clone(), r.n_contrib.clone())
    r2, _, _ = gpu_render(s)
    r2.render(*_params(P), mesh)
    torch.cuda.synchronize()
    assert torch.equal(got[0], r2.rgb)
    assert torch.equal(got[1], r2.T)
    assert torch.equal(got[2], r2.n_contrib)


def test_autotune_covers_the_grid_and_does_not_change_the_image():
    s = _room(seed=33, res=((160, 120), (96, 64)))
    g = s.gaussians
    P = gaussians_to_torch(g)
    mesh = MeshInput.from_numpy(s.mesh)
    kw = dict(sh_f16=True, n_verts=len(s.mesh.verts), n_faces=len(s.mesh.faces),
              tex_shape=s.mesh.texture.shape, bg=tuple(np.asarray(s.bg, np.float64)))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    npix = sum(c.width * c.height for c in s.cameras)
    dI = torch.randn(3 * npix, device="cuda", generator=gen)
    res = autotune.tune(s.cameras, g.n, g.sh_degree, _params(P), mesh, dL_drgb=dI, tex_grad=True,
                        warmup=1, iters=2, **kw)
    combos = {(t, b, p) for t, b, p, _ in res.table}
    want = {((16, 16), b) for b in (32, 64, 128, 256)} | {((32, 8), b) for b in (32, 64, 128, 256)} \
        | {((8, 8), b) for b in (32, 64)}
    assert combos == {(t, b, p) for t, b in want for p in (False, True)}
    assert all(np.isfinite(ms) and ms > 0 for _, _, _, ms in res.table)
    assert (res.tile, res.batch, res.persistent) in combos
    ref, _, _ = gpu_render(s)
    r = res.renderer
    r.render(*_params(P), mesh)
    torch.cuda.synchronize()
    assert torch.equal(r.rgb, ref.rgb)
    assert torch.equal(r.T, ref.T)
    assert torch.equal(r.n_contrib, ref.n_contrib)


@pytest.mark.parametrize("tile,batch,persistent", [((16, 16), 32, False), ((32, 8), 128, False), ((8, 8), 64, False),
                                                   ((16, 16), 128, True), ((8, 8), 32, True)])
def test_batched_uneven_fp16_backward_matches_oracle(tile, batch, persistent):
    s = _room(seed=34)
    rng = np.random.default_rng(7)
    gI_views, gT_views = [], []
    ref = None
    for v, cam in enumerate(s.cameras):
        npx = cam.n_pixels
        gI = rng.standard_normal((3, npx))
        gT = rng.standard_normal(npx)
        amb = O.render(s, view=v).out.amb
        gI[:, amb] = 0.0
        gT[amb] = 0.0
        _, gv = TR.render_grad(s, v, gI, gT)
        ref = gv if ref is None else {k: ref[k] + gv[k] for k in ref}
        gI_views.append(gI)
        gT_views.append(gT)
    r, P, mesh = gpu_render(s, tile=tile, batch=batch, persistent=persistent)
    dI = torch.as_tensor(np.concatenate([g.reshape(-1) for g in gI_views]), dtype=torch.float32, device="cuda")
    dT = torch.as_tensor(np.concatenate(gT_views), dtype=torch.float32, device="cuda")
    g = r.backward(*_params(P), dI, dT, mesh=mesh, tex_grad=True)
    torch.cuda.synchronize()
    for k in ("means", "scales", "quats", "opacity", "sh"):
        check_grad(k, g[k].cpu().numpy(), ref[k])
    gt = g["texture"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gt - ref["texture"]) <= 1e-3 * np.linalg.norm(ref["texture"])


def test_chunked_renderer_recomputes_lists_and_matches_the_batched_renderer():
    """Cameras rendered two at a time through one scratch, lists recomputed in
    the backward: same images (bit-exact) and gradients (up to atomic order)
    as the renderer that keeps every view's lists."""
    from paper_2506_06988_b300.render import ChunkedRenderer
    res = ((160, 120), (160, 120), (96, 64), (160, 120), (160, 120))
    s = _room(seed=35, res=res)
    r, P, mesh = gpu_render(s)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    dI = torch.randn(3 * r.npix, device="cuda", generator=gen)
    dT = torch.randn(r.npix, device="cuda", generator=gen)
    ref_g = r.backward(*_params(P), dI, dT, mesh=mesh, tex_grad=True)
    g = s.gaussians
    cr = ChunkedRenderer(s.cameras, g.n, g.sh_degree, chunk=2, sh_f16=True, n_verts=len(s.mesh.verts),
                         n_faces=len(s.mesh.faces), tex_shape=s.mesh.texture.shape,
                         bg=tuple(np.asarray(s.bg, np.float64)))
    cr.render(*_params(P), mesh)
    torch.cuda.synchronize()
    assert len(cr._renderers) == 3      # size patterns (160,160), (96,160), (160,)
    # (last_idx is a position in the renderer's own pair list, so it differs)
    for k in ("rgb", "T", "n_contrib", "tri_id", "mesh_depth", "mesh_rgb", "uv"):
        assert torch.equal(getattr(cr, k), getattr(r, k)), k
    got = cr.backward(*_params(P), dI, dT, mesh=mesh, tex_grad=True)
    assert cr.status() == 0
    _grads_close(got, ref_g)


def test_stream_overlap_gives_the_sequential_results():
    """The mesh pass on a side stream beside the projection and the binning
    (then without the tile mesh cull), and the texel gradients beside the
    blend and projection gradients: the same images, counts and stop indices
    (bit-exact) and gradients (up to atomic order) as one stream."""
    s = _room(seed=36)
    r, P, mesh = gpu_render(s)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(6)
    dI = torch.randn(3 * r.npix, device="cuda", generator=gen)
    r.forward(*_params(P), mesh, overlap=False)
    seq = {k: getattr(r, k).clone() for k in ("rgb", "T", "n_contrib", "mesh_depth", "tri_id", "mesh_rgb",
                                               "uv", "tile_max")}
    g_seq = r.backward(*_params(P), dI, None, mesh=mesh, tex_grad=True, overlap=False)
    r.forward(*_params(P), mesh, overlap=True)
    g_ovl = r.backward(*_params(P), dI, None, mesh=mesh, tex_grad=True, overlap=True)
    torch.cuda.synchronize()
    for k, v in seq.items():
        assert torch.equal(getattr(r, k), v), k
    _grads_close(g_ovl, g_seq)


@pytest.mark.parametrize("tile,batch", [((16, 16), 128), ((32, 8), 64), ((8, 8), 32)])
def test_persistent_launch_matches_grid_launch_and_oracle(tile, batch):
    """The (view, tile) work-queue launch of the blend kernels over three
    cameras of uneven size: the grid launch's outputs bit for bit, the same
    gradients up to FP32 atomic order, and the oracle's images."""
    s = _room(seed=35)
    a, P, mesh = gpu_render(s, tile=tile, batch=batch)
    b, _, _ = gpu_render(s, tile=tile, batch=batch, persistent=True)
    assert b.status()[0] == 0
    for k in ("rgb", "T", "n_contrib", "last_idx"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    for v in range(len(s.cameras)):
        compare_blend(view_outputs(b, v), oracle_view(s, v))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    dI = torch.randn(3 * a.npix, device="cuda", generator=gen)
    ga = a.backward(*_params(P), dI, None, mesh=mesh, tex_grad=True)
    gb = b.backward(*_params(P), dI, None, mesh=mesh, tex_grad=True)
    torch.cuda.synchronize()
    assert b.status()[0] == 0
    _grads_close(gb, ga)
