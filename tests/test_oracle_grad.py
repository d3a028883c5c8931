"""Pin of the FP64 gradient oracle (torch_ref, autograd through the plain
restatement of the forward) against central finite differences of the
independent C forward (hm_oracle.c), in FP64 (no GPU), step 1e-5 relative.

The derivative is of the hybrid composite of Sec. 3.4 (I_h = I_gs + T I_m)
built on Eq. 2, with respect to the Gaussian parameters and the texels (the
texture map is optimisable, Sec. 3.4).  Samples whose +-h perturbation flips
any discrete decision (blended set, alpha clamp, colour clamp, visibility)
are discarded, since the derivative does not exist there.
"""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import oracle as O
from oracle import torch_ref as TR
from paper_2506_06988_b300 import scenes


def _as64(g):
    return SimpleNamespace(means=np.array(g.means, np.float64), scales=np.array(g.scales, np.float64),
                           quats=np.array(g.quats, np.float64), opacity=np.array(g.opacity, np.float64),
                           sh=np.array(g.sh, np.float64), sh_degree=g.sh_degree)


def _loss(scene, g, tex, gI, gT, flt):
    r = O.render(scene, gaussians=g, tex=tex, **flt)
    L = float((r.out.rgb * gI).sum() + (r.out.T * gT).sum())
    key = (r.out.fp.tobytes(), r.proj.clamped.tobytes(), r.proj.visible.tobytes())
    return L, key


def _check(scene, n_per_kind, seed, rtol=2e-5, flt=None):
    """``flt``: projection filter options (the Mip-Splatting ones) passed to
    both oracles."""
    flt = dict(flt or {})
    rng = np.random.default_rng(seed)
    cam = scene.cameras[0]
    npx = cam.n_pixels
    gI = rng.standard_normal((3, npx))
    gT = rng.standard_normal(npx)
    g = _as64(scene.gaussians)
    tex = O.texture_unit(scene.mesh.texture).copy() if scene.mesh is not None else None
    _, grads = TR.render_grad(scene, 0, gI, gT, gaussians=g, tex=tex, **flt)
    base = O.render(scene, gaussians=g, tex=tex, **flt)
    # Gaussians that are blended somewhere (non-trivial gradients)
    contributing = np.nonzero(np.abs(grads["opacity"]) > 1e-3)[0]
    assert len(contributing) > 20
    checked = 0
    worst = 0.0
    kinds = [("means", 3), ("scales", 3), ("quats", 4), ("opacity", 0), ("sh", -1)]
    if tex is not None:
        kinds.append(("texture", -2))
    for name, width in kinds:
        for _ in range(n_per_kind):
            if name == "texture":
                tg = np.abs(grads["texture"]).reshape(-1)
                cand = np.nonzero(tg > 1e-3)[0]
                flat = int(rng.choice(cand))
                arr = tex
                idx = np.unravel_index(flat, tex.shape)
            else:
                i = int(rng.choice(contributing))
                arr = getattr(g, name)
                if width == 0:
                    idx = (i,)
                elif width == -1:
                    idx = (i, int(rng.integers(0, arr.shape[1])), int(rng.integers(0, 3)))
                else:
                    idx = (i, int(rng.integers(0, width)))
            v0 = arr[idx]
            # central differences: truncation O(h^2) ~ 1e-10 relative; round-off
            # |dL| / h with |dL| ~ 1e-13 for this loss stays ~1e-8 at h = 1e-5 |v|
            h = 1e-5 * max(abs(v0), 1e-2)
            arr[idx] = v0 + h
            Lp, kp = _loss(scene, g, tex, gI, gT, flt)
            arr[idx] = v0 - h
            Lm, km = _loss(scene, g, tex, gI, gT, flt)
            arr[idx] = v0
            k0 = (base.out.fp.tobytes(), base.proj.clamped.tobytes(), base.proj.visible.tobytes())
            if kp != k0 or km != k0:
                continue                      # a discrete decision flips inside +-h
            fd = (Lp - Lm) / (2 * h)
            ad = grads[name][idx]
            err = abs(fd - ad)
            tol = rtol * abs(ad) + 1e-6
            worst = max(worst, err / (abs(ad) + 1e-12))
            assert err <= tol, (name, idx, fd, ad)
            checked += 1
    return checked, worst


def test_gradient_oracle_matches_finite_differences_hybrid_sh0():
    """Config-0 hybrid scene (quad at z=3, SH degree 0): 64 parameters."""
    s = scenes.config0_scene(seed=0)
    s.bg = np.array([0.2, 0.3, 0.4], np.float32)
    checked, worst = _check(s, n_per_kind=11, seed=1)
    assert checked >= 50


def test_gradient_oracle_matches_finite_differences_sh3_no_mesh():
    """Degree-3 SH (view-dependent colour, gradient through the view
    direction into the means), Gaussian-only with a non-black background."""
    s = scenes.config0_scene(seed=2, n=600)
    rng = np.random.default_rng(5)
    g = s.gaussians
    g.sh = rng.normal(0.0, 0.2, (g.n, 16, 3)).astype(np.float32)
    g.sh_degree = 3
    s.mesh = None
    s.bg = np.array([0.5, 0.25, 0.1], np.float32)
    checked, worst = _check(s, n_per_kind=13, seed=3)
    assert checked >= 50
