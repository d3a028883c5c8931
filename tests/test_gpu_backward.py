"""GPU gradients (hm_blend_backward through the C ABI, and the autograd
Function on top) against the FP64 gradient oracle (autograd through the
plain restatement, itself pinned to finite differences of the C oracle).

Relative error bound 1e-3: per gradient tensor, ||g_gpu - g_ref|| <= 1e-3
||g_ref||, and per element |g_gpu - g_ref| <= 1e-3 |g_ref| + 1e-4 max|g_ref|
(the floor absorbs FP32 atomic accumulation order on near-cancelling sums).
Pixels whose forward decisions are ambiguous between FP32 and FP64 get a zero
upstream gradient, so both sides differentiate the same discrete branch."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import torch_ref as TR
from paper_2506_06988_b300 import lib, scenes
from paper_2506_06988_b300.render import HybridRender, MeshInput

from gpu_util import check_grad, gpu_render, gaussians_to_torch, make_renderer  # noqa: E402

pytestmark = pytest.mark.gpu


def _check(name, g, ref, rel=1e-3, floor=1e-4):
    return check_grad(name, g, ref, rel, floor)


def _run(scene, tex_grad, seed=0, tile=(16, 16), batch=None):
    cam = scene.cameras[0]
    npx = cam.n_pixels
    rng = np.random.default_rng(seed)
    gI = rng.standard_normal((3, npx))
    gT = rng.standard_normal(npx)
    orc = O.render(scene)
    amb = orc.out.amb
    gI[:, amb] = 0.0
    gT[amb] = 0.0
    tex = O.texture_unit(scene.mesh.texture) if scene.mesh is not None else None
    _, ref = TR.render_grad(scene, 0, gI, gT, tex=tex)
    r, P, mesh = gpu_render(scene, tile=tile, batch=batch)
    g = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"],
                   torch.as_tensor(gI.reshape(-1), dtype=torch.float32, device="cuda"),
                   torch.as_tensor(gT, dtype=torch.float32, device="cuda"), mesh=mesh, tex_grad=tex_grad)
    torch.cuda.synchronize()
    errs = {}
    for k in ("means", "scales", "quats", "opacity", "sh"):
        errs[k] = _check(k, g[k].cpu().numpy(), ref[k])
    if tex_grad:
        # (a) against the oracle: norm-relative only -- the GPU's UVs are FP32
        # (half an ulp of u is ~6e-5 texel at 2048 texels), which moves
        # individual bilinear weights by that much
        gt = g["texture"].cpu().numpy().astype(np.float64)
        errs["texture"] = float(np.linalg.norm(gt - ref["texture"]) / np.linalg.norm(ref["texture"]))
        assert errs["texture"] <= 1e-3, errs
        # (b) the texel scatter itself, exactly: FP64 scatter of T * w * dL/dI
        # from the GPU's own uv and T
        uv = r.uv.view(2, -1).cpu().numpy().astype(np.float64)
        T = r.T.cpu().numpy().astype(np.float64)
        hit = np.isfinite(r.mesh_depth.cpu().numpy())
        th, tw = scene.mesh.texture.shape[:2]
        want = np.zeros((th, tw, 3))
        s_ = uv[0] * np.float32(tw) - 0.5
        t_ = uv[1] * np.float32(th) - 0.5
        x0, y0 = np.floor(s_), np.floor(t_)
        fx, fy = s_ - x0, t_ - y0
        for dx, dy, w in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)), (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
            xi = np.clip(x0 + dx, 0, tw - 1).astype(np.int64)
            yi = np.clip(y0 + dy, 0, th - 1).astype(np.int64)
            for ch in range(3):
                np.add.at(want[:, :, ch], (yi[hit], xi[hit]), (T * w * gI[ch])[hit])
        _check("texture_scatter", gt, want, rel=1e-4, floor=1e-6)
    return errs


def test_backward_config0_hybrid_with_texture():
    s = scenes.config0_scene(seed=0)
    s.bg = np.array([0.2, 0.3, 0.4], np.float32)
    print(_run(s, tex_grad=True))


def test_backward_sh3_gaussian_only():
    s = scenes.config0_scene(seed=2, n=800)
    rng = np.random.default_rng(5)
    s.gaussians.sh = rng.normal(0.0, 0.2, (s.gaussians.n, 16, 3)).astype(np.float32)
    s.gaussians.sh_degree = 3
    s.mesh = None
    s.bg = np.array([0.5, 0.25, 0.1], np.float32)
    print(_run(s, tex_grad=False, seed=1))


def test_backward_room_sh3_hybrid():
    s = scenes.room_scene(21, n_tris=3000, n_gauss=5000, resolutions=((128, 96),))
    print(_run(s, tex_grad=True, seed=2))


@pytest.mark.parametrize("tile,batch", [((16, 16), 32), ((16, 16), 256), ((32, 8), 64), ((8, 8), 64)])
def test_backward_tile_shapes_and_batches(tile, batch):
    # every launch shape of the replay (two pixel pairs per thread on 16x16
    # tiles, one elsewhere; staged rounds of 32 to 256 records) on a view
    # whose size is no multiple of the tile (ragged right and bottom tiles)
    s = scenes.room_scene(22, n_tris=3000, n_gauss=5000, resolutions=((120, 90),))
    print(_run(s, tex_grad=True, seed=3, tile=tile, batch=batch))


def test_autograd_function_matches_direct_backward():
    """HybridRender (torch.autograd.Function) with activations in PyTorch:
    gradients of an L1 loss equal the direct C-ABI backward chained through
    exp/sigmoid by hand."""
    s = scenes.config0_scene(seed=1)
    s.mesh.texture = s.mesh.texture.astype(np.float32) / 255.0
    r = make_renderer(s)
    P = gaussians_to_torch(s.gaussians)
    mesh = MeshInput.from_numpy(s.mesh)
    log_s = torch.log(P["scales"]).requires_grad_()
    logit = torch.logit(P["opacity"]).requires_grad_()
    means = P["means"].clone().requires_grad_()
    quats = P["quats"].clone().requires_grad_()
    sh = P["sh"].clone().requires_grad_()
    tex = mesh.texture.clone().requires_grad_()
    target = torch.rand(3 * s.cameras[0].n_pixels, device="cuda")
    rgb, T = HybridRender.apply(r, mesh, means, torch.exp(log_s), quats, torch.sigmoid(logit), sh, tex)
    loss = (rgb - target).abs().mean()
    loss.backward()
    dI = torch.sign(rgb.detach() - target) / rgb.numel()
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], MeshInput(mesh.verts, mesh.uvs, mesh.faces, tex.detach()))
    g = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], dI, None,
                   mesh=MeshInput(mesh.verts, mesh.uvs, mesh.faces, tex.detach()), tex_grad=True)
    torch.testing.assert_close(means.grad, g["means"], rtol=1e-5, atol=1e-9)
    torch.testing.assert_close(log_s.grad, g["scales"] * P["scales"], rtol=1e-5, atol=1e-9)
    op = P["opacity"]
    torch.testing.assert_close(logit.grad, g["opacity"] * op * (1 - op), rtol=1e-5, atol=1e-9)
    torch.testing.assert_close(tex.grad, g["texture"], rtol=1e-5, atol=1e-9)


def test_config1_full_size_backward_sampled_pixels():
    """The bench workload (8 x 1920x1080, 300k Gaussians SH3, 50k-face room,
    texel gradients) in the bench's launch configuration (one GraphStep
    replay with the side-stream overlaps), with an upstream gradient on 64
    random unambiguous pixels of one view: every Gaussian parameter and texel
    gradient against the FP64 gradient oracle restricted to those pixels."""
    from paper_2506_06988_b300.render import GraphStep
    s = scenes.config1_scene()
    v = 1                                  # a pose facing the furniture: ~60 % of its pixels blend Gaussians
    r, P, mesh = gpu_render(s, tile=(16, 16))
    rng = np.random.default_rng(12)
    cand = np.sort(rng.choice(s.cameras[v].n_pixels, 4000, replace=False))
    orc = O.render(s, v, pix=cand)
    # unambiguous pixels where Gaussians are blended (most wall pixels have none)
    pix = cand[(~orc.out.amb) & (orc.out.n_contrib > 0)][:64]
    assert len(pix) == 64
    gI = rng.standard_normal((3, len(pix)))
    dI = np.zeros((3 * r.npix,), np.float64)
    a = int(r.pix_off[v])
    npx = s.cameras[v].n_pixels
    for c in range(3):
        dI[3 * a + c * npx + pix] = gI[c]
    tex = O.texture_unit(s.mesh.texture)
    _, ref = TR.render_grad(s, v, gI, None, pix=pix, tex=tex)
    dI_t = torch.as_tensor(dI, dtype=torch.float32, device="cuda")
    gs = GraphStep(r, (P["means"], P["scales"], P["quats"], P["opacity"], P["sh"]), mesh, dL_drgb=dI_t,
                   tex_grad=True)
    gs.replay(check=True)
    torch.cuda.synchronize()
    g = gs.grads
    for k in ("means", "scales", "quats", "opacity", "sh"):
        _check(k, g[k].cpu().numpy(), ref[k])
    gt = g["texture"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gt - ref["texture"]) <= 1e-3 * np.linalg.norm(ref["texture"])


def test_texel_gradients_keep_relative_accuracy_across_1e6_of_range():
    """dL/dI_h spanning six decades inside every tile (log-uniform
    magnitudes, random signs): each texel gradient within 1e-3 relative of
    an FP64 scatter of the same inputs (the kernel's own uv, T and dL/dI),
    element by element with no floor scaled by the largest gradient."""
    s = scenes.config0_scene()
    s.mesh.texture = s.mesh.texture.astype(np.float32) / 255.0
    r, P, mesh = gpu_render(s)
    rng = np.random.default_rng(9)
    mag = 10.0 ** rng.uniform(-6.0, 0.0, (3, r.npix))
    dI_np = (mag * rng.choice([-1.0, 1.0], (3, r.npix))).astype(np.float32)
    dI = torch.as_tensor(dI_np.reshape(-1), device="cuda")
    g = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], dI, mesh=mesh, tex_grad=True,
                   stages=lib.HM_BWD_TEXTURE)
    torch.cuda.synchronize()
    got = g["texture"].cpu().numpy().astype(np.float64)
    th, tw = s.mesh.texture.shape[:2]
    uv = r.uv.view(2, -1).cpu().numpy().astype(np.float64)
    T = r.T.cpu().numpy().astype(np.float64)
    hit = np.isfinite(r.mesh_depth.cpu().numpy())
    # FP64 scatter with the kernel's FP32 footprint (the same texel indices
    # and weights): texel centres at half-integers, clamp to the edge
    ss = (uv[0] * np.float32(tw)).astype(np.float32) - np.float32(0.5)
    tt = (uv[1] * np.float32(th)).astype(np.float32) - np.float32(0.5)
    x0, y0 = np.floor(ss), np.floor(tt)
    fx, fy = (ss - x0).astype(np.float64), (tt - y0).astype(np.float64)
    want = np.zeros((th, tw, 3))
    sabs = np.zeros((th, tw, 3))                # sum of |taps| per texel
    ntap = np.zeros((th, tw, 3))                # taps per texel
    mtap = np.zeros((th, tw, 3))                # largest |tap| per texel
    gpx = T[None, :] * dI_np.astype(np.float64)
    for dx, dy, w in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)), (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
        xi = np.clip(x0 + dx, 0, tw - 1).astype(int)
        yi = np.clip(y0 + dy, 0, th - 1).astype(int)
        for c in range(3):
            np.add.at(want[:, :, c], (yi[hit], xi[hit]), (w * gpx[c])[hit])
            np.add.at(sabs[:, :, c], (yi[hit], xi[hit]), np.abs(w * gpx[c])[hit])
            np.add.at(ntap[:, :, c], (yi[hit], xi[hit]), (w != 0)[hit].astype(float))
            np.maximum.at(mtap[:, :, c], (yi[hit], xi[hit]), np.abs(w * gpx[c])[hit])
    nz = sabs != 0
    # 1e-3 of the texel's own gradient, plus the rounding of its own taps:
    # the kernel's per-texel fixed point (2^-20 of the texel's largest tap
    # over its channels, per tap) and the FP32 products -- nothing scaled by
    # other texels
    err = np.abs(got[nz] - want[nz])
    floor = (ntap * 2.0 ** -20 * mtap.max(2, keepdims=True))[nz] + 1e-6 * sabs[nz]
    assert (err <= 1e-3 * np.abs(want[nz]) + floor).all(), float((err / np.abs(want[nz])).max())
    assert (np.abs(want[nz]) < 1e-3 * sabs.max()).mean() > 0.05       # many texels far below the maximum
    assert not got[~nz].any()


def test_config1_full_size_colour_weights_telescope():
    """The blend replay and the texel gradients over every pixel of the
    8-view 1080p workload, pinned
    by an identity of Eq. 2: with dL/dI = (1, 0, 0) at every pixel and no
    dL/dT, each Gaussian's red-colour partial is the sum of its weights
    alpha_i T_i over the pixels that blended it, and those weights telescope
    per pixel to 1 - T_final (T_{i+1} = T_i (1 - alpha_i)).  So the partials
    of all records sum to sum_px (1 - T_px), while the green and blue
    partials are exactly 0.  The replay rebuilds every T_i from T_final by
    division, back to front, so a wrong stop position, a skipped or doubled
    entry or a wrong (1 - alpha) breaks the sum.  The partials are read from
    the backward workspace, whose first n_views * n * 9 floats hold them per
    record (dL/dcolour in columns 6-8)."""
    s = scenes.config1_scene()
    r, P, mesh = gpu_render(s, tile=(16, 16))
    dI = torch.zeros(3 * r.npix, device="cuda")       # planar per camera: [view][3][pixels]
    for v in range(r.V):
        a, b = int(r.pix_off[v]), int(r.pix_off[v + 1])
        dI[3 * a:3 * a + (b - a)] = 1.0
    g = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], dI, None,
                   mesh=mesh, tex_grad=True,
                   stages=lib.HM_BWD_BLEND | lib.HM_BWD_TEXTURE | lib.HM_BWD_PROJECT)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    M = r.V * r.n
    part = r.bwd_ws[: 4 * 9 * M].view(torch.float32).view(M, 9)
    want = float((1.0 - r.T.double()).sum())
    got = float(part[:, 6].double().sum())
    assert want > 0.02 * r.npix
    assert abs(got - want) <= 1e-4 * want, (got, want)
    assert not bool(part[:, 7:9].any())
    # the texels: I_h = ... + T I_m, and I_m is a bilinear mix whose four
    # weights sum to 1, so the red texel gradients sum to sum T over the
    # pixels the mesh covers; green and blue receive exactly 0
    dtex = g["texture"].reshape(-1, 3)
    want_t = float(r.T.double()[r.tri_id >= 0].sum())
    got_t = float(dtex[:, 0].double().sum())
    assert want_t > 0.5 * r.npix
    assert abs(got_t - want_t) <= 1e-5 * want_t, (got_t, want_t)
    assert not bool(dtex[:, 1:].any())
    # the projection backward: the red DC coefficient of a Gaussian gets
    # C0 = 1 / (2 sqrt(pi)) times the red partials of its records whose
    # colour max(0, 0.5 + SH) is not clamped (a clamped colour is exactly 0),
    # summed over the views -- a (Gaussian, view) pair the pair list missed
    # breaks the sum
    rec = r.records_view()
    live = rec[:, 8] > 0
    want_sh = 0.28209479177387814 * float(part[live, 6].double().sum())
    got_sh = float(g["sh"][:, 0, 0].double().sum())
    assert abs(got_sh - want_sh) <= 1e-5 * abs(want_sh) + 1e-6, (got_sh, want_sh)
    assert not bool(g["sh"][:, 0, 1:].any())
