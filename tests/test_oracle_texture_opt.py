"""Pins of the texture-optimisation oracle: Adam's closed forms (the first
step moves every parameter by lr g / (|g| + eps), a constant gradient keeps
the step at lr after bias correction), and texture recovery on a quad seen
head-on -- starting from grey, the fitted texels approach the texture that
rendered the targets."""
import numpy as np

from oracle import oracle as O
from oracle import texture_opt as TO
from paper_2506_06988_b300 import scenes


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    p1, m1, v1 = TO.adam_step(p, g, z, z, 1, lr=0.05, eps=1e-8)
    assert np.allclose(p1, p - 0.05 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # a constant gradient: m_hat = g, v_hat = g^2 at every step
    p2, _, _ = TO.adam_step(p1, g, m1, v1, 2, lr=0.05, eps=0.0)
    assert np.allclose(p2, p1 - 0.05 * np.sign(g), rtol=0, atol=1e-12)


def test_texture_recovery_on_a_quad():
    rng = np.random.default_rng(1)
    s = scenes.micro_quad_only(w=24, h=24, f=24.0)
    true_tex = rng.uniform(0.1, 0.9, (8, 8, 3))
    s.mesh.texture = true_tex.astype(np.float32)
    targets = [O.mesh_raster(c, s.mesh, bg=np.asarray(s.bg, np.float64), tex=true_tex).rgb.reshape(3, 24, 24)
               for c in s.cameras]
    tex = np.full_like(true_tex, 0.5)
    m = np.zeros_like(tex)
    v = np.zeros_like(tex)
    first = None
    for t in range(1, 61):
        terms, _, tex, m, v = TO.texture_step(s, targets, tex, m, v, t, lr=0.05)
        first = terms[3] if first is None else first
    assert terms[3] < 0.2 * first
    assert np.abs(tex - true_tex).mean() < 0.5 * np.abs(0.5 - true_tex).mean()
