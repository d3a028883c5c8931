"""Oracle of texture optimisation from images alone (TEST INFRASTRUCTURE ONLY).

Before the joint optimisation the paper initialises the texture map of the
pruned mesh under image supervision through a differentiable rasteriser
(Sec. 3.3, Algorithm 1 stage 1): the texels are fitted so that the mesh
render matches the training images.  Readings: the render is the mesh pass
alone (I = I_m where a triangle covers the pixel, the background elsewhere);
the loss is the photometric loss of Eq. 3 on it (0.8 L1 + 0.2 D-SSIM, as in
the joint optimisation); the texels are updated by Adam (Kingma and Ba,
2015): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

``adam_step`` is that update in FP64; ``texture_step`` one full step (render,
loss, texel gradient, update) built from the mesh oracle, the loss oracle and
the gradient oracle.
"""
from __future__ import annotations

import numpy as np

from oracle import loss as LO
from oracle import oracle as O
from oracle import torch_ref as TR


def adam_step(p, g, m, v, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (p, m, v), FP64."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def texture_step(scene, targets, tex, m, v, t, lr=1e-2, lambda_s=0.2):
    """One step over all cameras of ``scene`` (its Gaussians ignored).
    targets: per camera [3, H, W]; tex [Ht, Wt, 3] FP64 texels.  Returns
    (loss terms (L1, SSIM, L_t, L), gradient, new tex, m, v)."""
    views = []
    renders = []
    for k, cam in enumerate(scene.cameras):
        mr = O.mesh_raster(cam, scene.mesh, bg=np.asarray(scene.bg, np.float64), tex=tex)
        H, W = int(cam.height), int(cam.width)
        x = mr.rgb.reshape(3, H, W)
        renders.append(mr)
        views.append(dict(x=x, y=np.asarray(targets[k], np.float64), m=x, T=np.ones((H, W)),
                          hit=np.zeros((H, W), bool)))
    terms, gx, _ = LO.loss_and_grads(views, lambda_s=lambda_s, lambda_t=0.0)
    grad = np.zeros_like(tex)
    empty = _no_gaussians(scene)
    for k, cam in enumerate(scene.cameras):
        _, g = TR.render_grad(empty, k, gx[k].reshape(3, -1), None, tex=tex)
        grad += g["texture"]
    new_tex, m, v = adam_step(tex, grad, m, v, t, lr=lr)
    return terms, grad, new_tex, m, v


def _no_gaussians(scene):
    from types import SimpleNamespace
    g = SimpleNamespace(means=np.zeros((0, 3)), scales=np.zeros((0, 3)), quats=np.zeros((0, 4)),
                        opacity=np.zeros(0), sh=np.zeros((0, 1, 3)), sh_degree=0, n=0)
    return SimpleNamespace(cameras=scene.cameras, gaussians=g, mesh=scene.mesh, bg=scene.bg)
