"""FP64 oracle of the joint-optimisation loss (TEST INFRASTRUCTURE ONLY).

The paper supervises the hybrid render I_h with the photometric loss of
Eq. 3, L_c = (1 - lambda_s) L1(I, I_h) + lambda_s D-SSIM(I, I_h) with
lambda_s = 0.2, and the textured mesh with the transmittance-aware texture
loss of Sec. 3.4, L_t = M_T ||I~ - I~_m||^2 (Eq. 5) with the mask
M_T = 1 / (1 + exp(-k (T - 0.5))) (Eq. 6), k = 20, where I~ and I~_m are the
target and the mesh colour on pixels with a triangle and 0 elsewhere; the
joint loss is L = L_c + lambda_t L_t (Eq. 7) with lambda_t = 0.1
(supplementary implementation details).

Readings (the paper leaves them open):
* every term is a mean over all pixel-channel elements of all cameras;
* SSIM is the standard single-scale form with an 11 x 11 Gaussian window of
  sigma 1.5 (normalised over its 11 taps per axis), zero padding at the
  image border, C1 = 0.01^2, C2 = 0.03^2, and D-SSIM = 1 - mean SSIM;
* M_T is a mask: no gradient flows through T.

``loss_and_grads`` evaluates the loss with plain float64 tensor ops and
differentiates it with autograd; the window step is a float64 2D
convolution written out here (its pin is scipy's Gaussian filter).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64
WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gauss_taps(win: int = WIN, sigma: float = SIGMA) -> np.ndarray:
    """1D Gaussian weights on offsets -win//2 .. win//2, summing to 1."""
    k = np.arange(win, dtype=np.float64) - (win // 2)
    g = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return g / g.sum()


def window_mean(img: torch.Tensor) -> torch.Tensor:
    """Gaussian-window weighted sum of each pixel's neighbourhood, zero
    outside the image: img [C, H, W] float64 -> [C, H, W]."""
    g = torch.as_tensor(gauss_taps(), dtype=DT)
    w2 = torch.outer(g, g)[None, None].repeat(img.shape[0], 1, 1, 1)
    return torch.nn.functional.conv2d(img[None], w2, padding=WIN // 2, groups=img.shape[0])[0]


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Per-pixel SSIM of x against y ([C, H, W] float64)."""
    mx, my = window_mean(x), window_mean(y)
    sxx = window_mean(x * x) - mx * mx
    syy = window_mean(y * y) - my * my
    sxy = window_mean(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def loss_terms(views, lambda_s=0.2, lambda_t=0.1, k=20.0):
    """views: list of dicts with float64 tensors x (I_h), y (target),
    m (I_m) of shape [3, H, W], T [H, W] and hit [H, W] (bool).  Returns
    (L1, mean SSIM, L_t, L) over all pixel-channel elements of all views."""
    n = sum(v["x"].numel() for v in views)
    l1 = sum((v["x"] - v["y"]).abs().sum() for v in views) / n
    ss = sum(ssim_map(v["x"], v["y"]).sum() for v in views) / n
    lt = 0.0
    for v in views:
        mt = 1.0 / (1.0 + torch.exp(-k * (v["T"].detach() - 0.5)))
        hit = v["hit"].to(DT)
        d = hit * (v["y"] - v["m"])
        lt = lt + (mt * hit * (d * d).sum(0)).sum()
    lt = lt / n
    lc = (1.0 - lambda_s) * l1 + lambda_s * (1.0 - ss)
    return l1, ss, lt, lc + lambda_t * lt


def loss_and_grads(views_np, lambda_s=0.2, lambda_t=0.1, k=20.0):
    """views_np: list of dicts of numpy arrays (x, y, m [3,H,W]; T, hit
    [H,W]).  Returns (terms as floats, [dL/dx per view], [dL/dm per view])."""
    views = []
    for v in views_np:
        views.append(dict(x=torch.tensor(np.asarray(v["x"], np.float64), requires_grad=True),
                          y=torch.tensor(np.asarray(v["y"], np.float64)),
                          m=torch.tensor(np.asarray(v["m"], np.float64), requires_grad=True),
                          T=torch.tensor(np.asarray(v["T"], np.float64)),
                          hit=torch.tensor(np.asarray(v["hit"], bool))))
    l1, ss, lt, L = loss_terms(views, lambda_s, lambda_t, k)
    L.backward()
    terms = tuple(float(t.detach()) if torch.is_tensor(t) else float(t) for t in (l1, ss, lt, L))
    return terms, [v["x"].grad.numpy() for v in views], [v["m"].grad.numpy() for v in views]
