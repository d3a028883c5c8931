"""hm_hybrid_loss (Eq. 3 photometric loss with D-SSIM, the Sec. 3.4
transmittance-aware texture loss) against the FP64 loss oracle, and the
texel gradient of the joint loss through hm_blend_backward.

Tolerances: the loss terms are sums of FP32 per-pixel values accumulated in
FP64, relative 1e-5.  dL/dI_h is a difference of 11-tap window sums of
products (FP32, relative error ~1e-6 of the largest terms), checked as
||g - g_ref|| <= 1e-4 ||g_ref|| and per element within 1e-3 relative plus
1e-4 of the largest magnitude; dL/dI_m is pointwise, relative 1e-5."""
import numpy as np
import pytest
import torch

from oracle import loss as LO
from paper_2506_06988_b300 import lib, scenes
from paper_2506_06988_b300.render import MeshInput

from gpu_util import gaussians_to_torch, gpu_render  # noqa: E402

pytestmark = pytest.mark.gpu


def _case(rng, sizes):
    cams, views = [], []
    for w, h in sizes:
        cams.append(scenes._identity_cam(w, h))
        hit = rng.uniform(0, 1, (h, w)) < 0.7
        views.append(dict(x=rng.uniform(0, 1, (3, h, w)), y=rng.uniform(0, 1, (3, h, w)),
                          m=rng.uniform(0, 1, (3, h, w)), T=rng.uniform(0, 1, (h, w)), hit=hit))
    return cams, views


def _flat(views, key):
    return torch.as_tensor(np.concatenate([np.asarray(v[key], np.float32).reshape(-1) for v in views]),
                           device="cuda")


@pytest.mark.parametrize("sizes", [((37, 23),), ((16, 16), (5, 7), (70, 33)), ((100, 70), (33, 64))])
def test_hybrid_loss_matches_oracle(sizes):
    rng = np.random.default_rng(len(sizes))
    cams_np, views = _case(rng, sizes)
    cams = lib.cameras(cams_np)
    x, y, m = _flat(views, "x"), _flat(views, "y"), _flat(views, "m")
    T = _flat(views, "T")
    depth = torch.as_tensor(np.concatenate([np.where(v["hit"], 2.0, np.inf).reshape(-1) for v in views]),
                            dtype=torch.float32, device="cuda")
    # the oracle sees exactly the FP32 inputs
    for v in views:
        for k in ("x", "y", "m", "T"):
            v[k] = np.asarray(v[k], np.float32).astype(np.float64)
    (l1, ss, lt, L), gx, gm = LO.loss_and_grads(views, lambda_s=0.2, lambda_t=0.1, k=20.0)
    ws = torch.empty(lib.hm_hybrid_loss_workspace_size(cams), dtype=torch.uint8, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    dI = torch.empty_like(x)
    dM = torch.empty_like(x)
    lib.check(lib.hm_hybrid_loss(cams, x, y, m, T, depth, lib.loss_params(), out, dI, dM, ws, ws.numel(),
                                 torch.cuda.current_stream().cuda_stream), "hm_hybrid_loss")
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = np.array([l1, ss, lt, L])
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-9), (got, want)
    # the partial sums are reduced in a fixed order: a second call repeats every bit
    out2, dI2 = torch.empty_like(out), torch.empty_like(dI)
    lib.check(lib.hm_hybrid_loss(cams, x, y, m, T, depth, lib.loss_params(), out2, dI2, dM, ws, ws.numel(),
                                 torch.cuda.current_stream().cuda_stream), "hm_hybrid_loss")
    torch.cuda.synchronize()
    assert torch.equal(out, out2) and torch.equal(dI, dI2)
    g_ref = np.concatenate([g.reshape(-1) for g in gx])
    g = dI.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert np.all(np.abs(g - g_ref) <= 1e-3 * np.abs(g_ref) + 1e-4 * np.abs(g_ref).max())
    gm_ref = np.concatenate([gg.reshape(-1) for gg in gm])
    gmv = dM.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gmv - gm_ref) <= 1e-5 * np.abs(gm_ref) + 1e-12 * max(1.0, np.abs(gm_ref).max()))


def test_hybrid_loss_without_mesh_and_weights():
    rng = np.random.default_rng(9)
    cams_np, views = _case(rng, ((40, 30),))
    cams = lib.cameras(cams_np)
    x, y = _flat(views, "x"), _flat(views, "y")
    for v in views:
        v["x"] = np.asarray(v["x"], np.float32).astype(np.float64)
        v["y"] = np.asarray(v["y"], np.float32).astype(np.float64)
        v["hit"] = np.zeros_like(v["hit"])
    (l1, ss, lt, L), gx, _ = LO.loss_and_grads(views, lambda_s=0.5, lambda_t=0.3, k=20.0)
    ws = torch.empty(lib.hm_hybrid_loss_workspace_size(cams), dtype=torch.uint8, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    dI = torch.empty_like(x)
    lib.check(lib.hm_hybrid_loss(cams, x, y, None, None, None, lib.loss_params(lambda_ssim=0.5, lambda_t=0.3),
                                 out, dI, None, ws, ws.numel(), torch.cuda.current_stream().cuda_stream),
              "hm_hybrid_loss")
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[2] == 0.0 and lt == 0.0
    want = np.array([l1, ss, lt, L])
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-9), (got, want)
    g_ref = gx[0].reshape(-1)
    assert np.linalg.norm(dI.cpu().numpy() - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_joint_loss_texel_gradient_scatter():
    """Texels of the joint loss receive w (T dL/dI_h + dL/dI_m): checked
    exactly (FP64 scatter from the GPU's own uv, T and loss gradients)."""
    s = scenes.config0_scene(seed=4)
    s.mesh.texture = s.mesh.texture.astype(np.float32) / 255.0
    r, P, mesh = gpu_render(s)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(8)
    target = torch.rand(3 * r.npix, device="cuda", generator=gen)
    terms, dI, dM = r.loss(target)
    g = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], dI, None, mesh=mesh,
                   tex_grad=True, dL_dmesh=dM)
    torch.cuda.synchronize()
    assert np.isfinite(terms.cpu().numpy()).all()
    uv = r.uv.view(2, -1).cpu().numpy().astype(np.float64)
    T = r.T.cpu().numpy().astype(np.float64)
    hit = np.isfinite(r.mesh_depth.cpu().numpy())
    up = T * dI.view(3, -1).cpu().numpy().astype(np.float64) + dM.view(3, -1).cpu().numpy().astype(np.float64)
    th, tw = s.mesh.texture.shape[:2]
    want = np.zeros((th, tw, 3))
    s_ = uv[0] * np.float32(tw) - 0.5
    t_ = uv[1] * np.float32(th) - 0.5
    x0, y0 = np.floor(s_), np.floor(t_)
    fx, fy = s_ - x0, t_ - y0
    for dx, dy, w in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)), (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
        xi = np.clip(x0 + dx, 0, tw - 1).astype(np.int64)
        yi = np.clip(y0 + dy, 0, th - 1).astype(np.int64)
        for ch in range(3):
            np.add.at(want[:, :, ch], (yi[hit], xi[hit]), (w * up[ch])[hit])
    got = g["texture"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)
    assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-6 * np.abs(want).max())


@pytest.mark.parametrize("sizes", [((37, 23),), ((16, 16), (5, 7), (70, 33)), ((64, 48), (32, 20))])
def test_hybrid_loss_without_ssim_term(sizes):
    # lambda_ssim = 0 takes the pointwise pass: L1, L_t and L as the oracle's,
    # dL/dI_h = sign(x - y) / N exactly, mean SSIM reported as 0 (cameras
    # whose pixel counts are all multiples of 4 take the four-pixel path)
    rng = np.random.default_rng(20 + len(sizes))
    cams_np, views = _case(rng, sizes)
    cams = lib.cameras(cams_np)
    x, y, m, T = _flat(views, "x"), _flat(views, "y"), _flat(views, "m"), _flat(views, "T")
    x[::7] = y[::7]                      # ties: the subgradient 0
    depth = torch.as_tensor(np.concatenate([np.where(v["hit"], 2.0, np.inf).reshape(-1) for v in views]),
                            dtype=torch.float32, device="cuda")
    xs = x.cpu().numpy()
    off = 0
    for v in views:
        n = v["x"].size
        v["x"] = xs[off:off + n].reshape(v["x"].shape).astype(np.float64)
        off += n
        for k in ("y", "m", "T"):
            v[k] = np.asarray(v[k], np.float32).astype(np.float64)
    (l1, _, lt, L), gx, gm = LO.loss_and_grads(views, lambda_s=0.0, lambda_t=0.1, k=20.0)
    ws = torch.empty(lib.hm_hybrid_loss_workspace_size(cams), dtype=torch.uint8, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    dI, dM = torch.empty_like(x), torch.empty_like(x)
    lp = lib.loss_params(lambda_ssim=0.0, lambda_t=0.1)
    lib.check(lib.hm_hybrid_loss(cams, x, y, m, T, depth, lp, out, dI, dM, ws, ws.numel(),
                                 torch.cuda.current_stream().cuda_stream), "hm_hybrid_loss")
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[1] == 0.0
    want = np.array([l1, lt, L])
    assert np.all(np.abs(got[[0, 2, 3]] - want) <= 1e-5 * np.abs(want) + 1e-9), (got, want)
    g_ref = np.concatenate([g.reshape(-1) for g in gx])
    assert np.array_equal(dI.cpu().numpy(), g_ref.astype(np.float32))
    gm_ref = np.concatenate([gg.reshape(-1) for gg in gm])
    gmv = dM.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gmv - gm_ref) <= 1e-5 * np.abs(gm_ref) + 1e-12 * max(1.0, np.abs(gm_ref).max()))
