"""Texture optimisation from images alone (Sec. 3.3's texture
initialisation): hm_adam_update against the FP64 Adam of the oracle, one
full step (mesh-only render, Eq. 3 loss, texel gradient, update) against the
oracle's step, and recovery of a known texture on the GPU.

Tolerances: Adam in FP32 vs FP64: the moments within 4 FP32 ulps of their
terms' magnitude (b1 |m| + (1 - b1) |g|, etc.), the parameters within 1e-6
absolute plus 2e-7 relative (values of order 1); the step's loss terms 1e-5 relative, the texel
gradient 1e-3 of its norm (FP32 UVs move bilinear weights by ~1e-5), the
updated texels within 1e-5 where the gradient is not near zero (Adam's first
step is lr sign(g), so a texel whose gradient is within rounding of zero may
go either way)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import texture_opt as TO
from paper_2506_06988_b300 import lib, scenes
from paper_2506_06988_b300.render import MeshInput
from paper_2506_06988_b300.texture_opt import TextureOptimizer

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("offset", [0, 1])
def test_adam_update_matches_oracle(offset):
    rng = np.random.default_rng(3)
    n = 1003
    base = [rng.standard_normal(n + offset).astype(np.float32) for _ in range(4)]
    base[3] = np.abs(base[3])                                   # v >= 0
    dev = [torch.as_tensor(a, device="cuda")[offset:] for a in base]     # offset 1: unaligned, scalar path
    p, g, m, v = (a.clone() if i != 1 else a for i, a in enumerate(dev))
    ref = [a[offset:].astype(np.float64) for a in base]
    ulp4 = 4 * 2.0 ** -23
    for step in (1, 7):
        m_scale = 0.9 * np.abs(ref[2]) + 0.1 * np.abs(ref[1])
        v_scale = 0.999 * np.abs(ref[3]) + 0.001 * ref[1] ** 2 + 1e-12
        lib.check(lib.hm_adam_update(p, g, m, v, n, 0.01, 0.9, 0.999, 1e-8, step,
                                     torch.cuda.current_stream().cuda_stream), "hm_adam_update")
        # the oracle takes the hyper-parameters the kernel received (FP32 values)
        f32 = lambda x: float(np.float32(x))  # noqa: E731
        ref[0], ref[2], ref[3] = TO.adam_step(ref[0], ref[1], ref[2], ref[3], step, lr=f32(0.01), b1=f32(0.9),
                                              b2=f32(0.999), eps=f32(1e-8))
        torch.cuda.synchronize()
        assert np.all(np.abs(m.cpu().numpy() - ref[2]) <= ulp4 * m_scale + 1e-30)
        assert np.all(np.abs(v.cpu().numpy() - ref[3]) <= ulp4 * v_scale + 1e-30)
        assert np.all(np.abs(p.cpu().numpy() - ref[0]) <= 1e-6 + 2e-7 * np.abs(ref[0]))


def _quad_scene(seed=1, n=24, tex_n=8):
    rng = np.random.default_rng(seed)
    s = scenes.micro_quad_only(w=n, h=n, f=float(n))
    true_tex = rng.uniform(0.1, 0.9, (tex_n, tex_n, 3))
    s.mesh.texture = true_tex.astype(np.float32)
    return s, true_tex


def test_texture_step_matches_oracle():
    s = scenes.config0_scene(seed=2)
    rng = np.random.default_rng(4)
    tex0 = rng.uniform(0.2, 0.8, s.mesh.texture.shape).astype(np.float32)
    true_tex = O.texture_unit(s.mesh.texture)
    cam = s.cameras[0]
    target = O.mesh_raster(cam, s.mesh, bg=np.asarray(s.bg, np.float64), tex=true_tex).rgb
    target = target.reshape(3, cam.height, cam.width)
    s.mesh.texture = tex0
    mesh = MeshInput.from_numpy(s.mesh)
    opt = TextureOptimizer(s.cameras, mesh, torch.as_tensor(target.astype(np.float32).reshape(-1), device="cuda"),
                           lr=0.01, bg=tuple(np.asarray(s.bg, np.float64)))
    terms = opt.step()
    torch.cuda.synchronize()
    t64 = tex0.astype(np.float64)
    z = np.zeros_like(t64)
    want_terms, grad, new_tex, _, _ = TO.texture_step(s, [target.astype(np.float32).astype(np.float64)], t64, z, z,
                                                      1, lr=0.01)
    got = terms.cpu().numpy()
    assert np.all(np.abs(got[[0, 1, 3]] - np.array(want_terms)[[0, 1, 3]]) <= 1e-5 * np.abs(np.array(want_terms)[[0, 1, 3]]))
    g = opt.grads["texture"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - grad) <= 1e-3 * np.linalg.norm(grad)
    firm = np.abs(grad) > 1e-3 * np.abs(grad).max()
    assert firm.mean() > 0.3
    assert np.abs(opt.texture.cpu().numpy()[firm] - new_tex[firm]).max() < 1e-5


def test_texture_recovery_on_gpu():
    s, true_tex = _quad_scene()
    cam = s.cameras[0]
    target = O.mesh_raster(cam, s.mesh, bg=np.asarray(s.bg, np.float64), tex=true_tex).rgb.astype(np.float32)
    s.mesh.texture = np.full_like(true_tex, 0.5, dtype=np.float32)
    opt = TextureOptimizer(s.cameras, MeshInput.from_numpy(s.mesh), torch.as_tensor(target.reshape(-1), device="cuda"),
                           lr=0.05, bg=tuple(np.asarray(s.bg, np.float64)))
    first = float(opt.step()[3])
    last = opt.run(59)[3]
    assert last < 0.2 * first
    err = np.abs(opt.texture.cpu().numpy() - true_tex).mean()
    assert err < 0.5 * np.abs(0.5 - true_tex).mean()


def test_texture_graph_step_matches_eager():
    # the captured step replays the eager one: the same first loss bit for
    # bit, the same step count, and texels that agree after three steps up
    # to the order of the texel gradients' global additions
    s = scenes.config0_scene(seed=2)
    rng = np.random.default_rng(5)
    tex0 = rng.uniform(0.2, 0.8, s.mesh.texture.shape).astype(np.float32)
    true_tex = O.texture_unit(s.mesh.texture)
    cam = s.cameras[0]
    target = O.mesh_raster(cam, s.mesh, bg=np.asarray(s.bg, np.float64), tex=true_tex).rgb.astype(np.float32)
    s.mesh.texture = tex0
    tgt = torch.as_tensor(target.reshape(-1), device="cuda")
    bg = tuple(np.asarray(s.bg, np.float64))
    eager = TextureOptimizer(s.cameras, MeshInput.from_numpy(s.mesh), tgt, lr=0.01, bg=bg)
    graph = TextureOptimizer(s.cameras, MeshInput.from_numpy(s.mesh), tgt, lr=0.01, bg=bg).capture()
    firsts = []
    for _ in range(3):
        a = eager.step(check=True).clone()
        b = graph.step(check=True).clone()
        firsts.append((a, b))
    torch.cuda.synchronize()
    assert torch.equal(firsts[0][0], firsts[0][1])
    assert eager.t == 3 and graph.t == 3
    d = (eager.texture - graph.texture).abs()
    assert float(d.max()) <= 2 * 0.01 * 3
    assert float((d > 1e-5).float().mean()) <= 1e-2
