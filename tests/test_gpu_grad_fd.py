"""GPU gradients (hm_blend_backward through the C ABI) against FP64 central
finite differences of the C oracle's forward on the config-0 hybrid scene
(2,000 Gaussians, a textured quad at z = 3, 128 x 128): 64 sampled
parameters over the means, scales, quaternions, opacities, SH coefficients
and FP32 texels (the texture is optimisable, Sec. 3.4).

L = sum_p gI[:, p] . I_h(p) + gT[p] T(p) with seeded gI, gT; pixels whose
forward decisions are ambiguous between FP32 and FP64 get zero upstream
gradient.  A sample whose +-h perturbation flips any discrete decision of
the oracle (the blended set, a clamp, visibility) is discarded -- the
derivative does not exist there.  Bound: |g_gpu - fd| <= 1e-3 |fd| plus a
floor of 1e-4 of the largest |gradient| of that parameter kind (FP32
accumulation of many near-cancelling terms).
"""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_06988_b300 import scenes
from paper_2506_06988_b300.render import MeshInput

from gpu_util import gaussians_to_torch, make_renderer  # noqa: E402

pytestmark = pytest.mark.gpu


def _loss(scene, g, tex, gI, gT):
    r = O.render(scene, gaussians=g, tex=tex)
    L = float((r.out.rgb * gI).sum() + (r.out.T * gT).sum())
    key = (r.out.fp.tobytes(), r.proj.clamped.tobytes(), r.proj.visible.tobytes())
    return L, key


def test_gpu_gradients_match_oracle_finite_differences_config0():
    s = scenes.config0_scene(seed=0)
    s.bg = np.array([0.2, 0.3, 0.4], np.float32)
    tex64 = O.texture_unit(s.mesh.texture).copy()
    s.mesh.texture = tex64.astype(np.float32)           # FP32 learnable texels on both sides
    tex64 = s.mesh.texture.astype(np.float64)
    cam = s.cameras[0]
    npx = cam.n_pixels
    rng = np.random.default_rng(11)
    gI = rng.standard_normal((3, npx))
    gT = rng.standard_normal(npx)
    base = O.render(s, tex=tex64)
    amb = base.out.amb
    gI[:, amb] = 0.0
    gT[amb] = 0.0

    r = make_renderer(s)
    P = gaussians_to_torch(s.gaussians)
    mesh = MeshInput.from_numpy(s.mesh)
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)
    dI = torch.as_tensor(gI.reshape(-1), dtype=torch.float32, device="cuda")
    dT = torch.as_tensor(gT, dtype=torch.float32, device="cuda")
    grads = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], dI, dT, mesh=mesh,
                       tex_grad=True)
    torch.cuda.synchronize()
    G = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}

    g64 = SimpleNamespace(means=np.array(s.gaussians.means, np.float64),
                          scales=np.array(s.gaussians.scales, np.float64),
                          quats=np.array(s.gaussians.quats, np.float64),
                          opacity=np.array(s.gaussians.opacity, np.float64),
                          sh=np.array(s.gaussians.sh, np.float64), sh_degree=s.gaussians.sh_degree)
    k0 = (base.out.fp.tobytes(), base.proj.clamped.tobytes(), base.proj.visible.tobytes())
    contributing = np.nonzero(np.abs(G["opacity"]) > 1e-3)[0]
    assert len(contributing) > 20
    kinds = [("means", 3), ("scales", 3), ("quats", 4), ("opacity", 0), ("sh", -1), ("texture", -2)]
    checked, tried, worst = 0, 0, 0.0
    while checked < 64:
        tried += 1
        assert tried < 400, (checked, tried)
        name, width = kinds[tried % len(kinds)]
        if name == "texture":
            cand = np.nonzero(np.abs(G["texture"]).reshape(-1) > 1e-3)[0]
            idx = np.unravel_index(int(rng.choice(cand)), tex64.shape)
            arr = tex64
        else:
            i = int(rng.choice(contributing))
            arr = getattr(g64, name)
            if width == 0:
                idx = (i,)
            elif width == -1:
                idx = (i, int(rng.integers(0, arr.shape[1])), int(rng.integers(0, 3)))
            else:
                idx = (i, int(rng.integers(0, width)))
        v0 = arr[idx]
        h = 1e-5 * max(abs(v0), 1e-2)
        arr[idx] = v0 + h
        Lp, kp = _loss(s, g64, tex64, gI, gT)
        arr[idx] = v0 - h
        Lm, km = _loss(s, g64, tex64, gI, gT)
        arr[idx] = v0
        if kp != k0 or km != k0:
            continue
        fd = (Lp - Lm) / (2 * h)
        got = G[name][idx]
        floor = 1e-4 * np.abs(G[name]).max()
        assert abs(got - fd) <= 1e-3 * abs(fd) + floor, (name, idx, got, fd)
        worst = max(worst, abs(got - fd) / (abs(fd) + 1e-12))
        checked += 1
    print("checked", checked, "tried", tried, "worst rel", worst)
