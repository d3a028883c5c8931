"""Pins of the FP64 loss oracle (Eq. 3 photometric loss with D-SSIM, the
Sec. 3.4 transmittance-aware texture loss) against facts that do not come
from the oracle itself: scipy's Gaussian filter for the SSIM window, the
closed forms of SSIM for identical and for constant images, the closed forms
of L1 and of L_t with a constant transmittance, and central finite
differences of the loss for the gradients."""
import numpy as np
import scipy.ndimage as ndi
import torch

from oracle import loss as LO


def _views(rng, shapes=((10, 12), (7, 9))):
    out = []
    for h, w in shapes:
        out.append(dict(x=rng.uniform(0, 1, (3, h, w)), y=rng.uniform(0, 1, (3, h, w)),
                        m=rng.uniform(0, 1, (3, h, w)), T=rng.uniform(0, 1, (h, w)),
                        hit=rng.uniform(0, 1, (h, w)) < 0.7))
    return out


def test_window_is_scipy_gaussian_filter():
    rng = np.random.default_rng(0)
    img = rng.uniform(0, 1, (3, 17, 23))
    got = LO.window_mean(torch.tensor(img)).numpy()
    for c in range(3):
        want = ndi.gaussian_filter(img[c], sigma=1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)
        assert np.abs(got[c] - want).max() < 1e-12


def test_ssim_of_identical_images_is_one_and_symmetric():
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.uniform(0, 1, (3, 16, 20)))
    y = torch.tensor(rng.uniform(0, 1, (3, 16, 20)))
    assert torch.allclose(LO.ssim_map(x, x), torch.ones_like(x), atol=1e-12)
    assert torch.allclose(LO.ssim_map(x, y), LO.ssim_map(y, x), atol=1e-14)


def test_ssim_of_constant_images_closed_form():
    a, b = 0.3, 0.8
    x = torch.full((3, 24, 24), a, dtype=torch.float64)
    y = torch.full((3, 24, 24), b, dtype=torch.float64)
    s = LO.ssim_map(x, y)[:, 5:-5, 5:-5]        # windows fully inside the image
    want = (2 * a * b + LO.C1) / (a * a + b * b + LO.C1)
    assert torch.allclose(s, torch.full_like(s, want), atol=1e-12)


def test_l1_and_texture_loss_closed_forms():
    rng = np.random.default_rng(2)
    vs = _views(rng)
    T0 = 0.62
    for v in vs:
        v["T"] = np.full_like(v["T"], T0)
    (l1, ss, lt, L), _, _ = LO.loss_and_grads(vs, lambda_s=0.2, lambda_t=0.1, k=20.0)
    n = sum(v["x"].size for v in vs)
    assert abs(l1 - sum(np.abs(v["x"] - v["y"]).sum() for v in vs) / n) < 1e-12
    mt = 1.0 / (1.0 + np.exp(-20.0 * (T0 - 0.5)))
    lt_want = sum((v["hit"][None] * (v["y"] - v["m"]) ** 2).sum() for v in vs) * mt / n
    assert abs(lt - lt_want) < 1e-12
    assert abs(L - (0.8 * l1 + 0.2 * (1 - ss) + 0.1 * lt)) < 1e-12


def test_loss_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    vs = _views(rng)
    _, gx, gm = LO.loss_and_grads(vs)
    checked = 0
    for _ in range(40):
        vi = int(rng.integers(0, len(vs)))
        name = "x" if rng.uniform() < 0.6 else "m"
        arr = vs[vi][name]
        idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
        v0 = arr[idx]
        h = 1e-6
        arr[idx] = v0 + h
        (_, _, _, Lp), _, _ = LO.loss_and_grads(vs)
        arr[idx] = v0 - h
        (_, _, _, Lm), _, _ = LO.loss_and_grads(vs)
        arr[idx] = v0
        fd = (Lp - Lm) / (2 * h)
        if abs(arr[idx] - vs[vi]["y"][idx]) < 1e-3 and name == "x":
            continue                       # |x - y| kink of L1 within reach
        ad = (gx if name == "x" else gm)[vi][idx]
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)) + 1e-8, (name, idx, fd, ad)
        checked += 1
    assert checked >= 30


def test_ssim_of_affinely_related_images_closed_form():
    """y = alpha x + beta: sigma_y^2 = alpha^2 sigma_x^2 and sigma_xy =
    alpha sigma_x^2, so SSIM reduces to a function of scipy-filtered mean
    and variance of x alone -- pins the cross term and the variance terms."""
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (1, 21, 19))
    alpha, beta = -0.6, 0.7
    y = alpha * x + beta
    f = lambda a: ndi.gaussian_filter(a, sigma=1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)  # noqa: E731
    mx = f(x[0])
    vx = f(x[0] * x[0]) - mx * mx
    # the window sums run over the zero padding too, so y's mean is
    # alpha mx + beta * (window mass inside the image)
    mass = f(np.ones_like(x[0]))
    my = alpha * mx + beta * mass
    vy = f(y[0] * y[0]) - my * my
    cxy = f(x[0] * y[0]) - mx * my
    inner = (slice(5, -5), slice(5, -5))       # mass = 1 there: vy = a^2 vx, cxy = a vx
    assert np.allclose(vy[inner], alpha ** 2 * vx[inner], atol=1e-12)
    assert np.allclose(cxy[inner], alpha * vx[inner], atol=1e-12)
    want = ((2 * mx * my + LO.C1) / (mx ** 2 + my ** 2 + LO.C1)
            * (2 * alpha * vx + LO.C2) / ((1 + alpha ** 2) * vx + LO.C2))
    got = LO.ssim_map(torch.tensor(x), torch.tensor(y)).numpy()[0]
    assert np.abs(got[inner] - want[inner]).max() < 1e-12


def test_transmittance_mask_special_values():
    """M_T is 1/2 at T = 1/2 and tends to 1 (mesh dominates) as T -> 1 and
    to 0 as T -> 0 (Sec. 3.4): L_t at those constant transmittances."""
    rng = np.random.default_rng(5)
    vs = _views(rng, shapes=((6, 8),))
    n = vs[0]["x"].size
    base = (vs[0]["hit"][None] * (vs[0]["y"] - vs[0]["m"]) ** 2).sum() / n
    for T0, scale in ((0.5, 0.5), (1.0, 1.0), (0.0, 0.0)):
        vs[0]["T"] = np.full_like(vs[0]["T"], T0)
        (_, _, lt, _), _, gm = LO.loss_and_grads(vs)
        assert abs(lt - scale * base) <= 5e-5 * base + 1e-15, (T0, lt, base)
