"""Pins of the oracle's Mip-Splatting filters (the second Gaussian back-end
the paper pairs with the mesh, Tab. 1; filters as published by Yu et al.,
CVPR 2024): the 3D smoothing-filter variance from the cameras' sampling
rates, the 3D filter and the 2D Mip filter in the projection, and the
gradient oracle with the filters on, against closed forms, the mass
conservation the opacity compensation exists for, and finite differences."""
from types import SimpleNamespace

import numpy as np

from oracle import oracle as O
from paper_2506_06988_b300 import scenes

from test_oracle_grad import _check  # noqa: E402


def _cam(f=100.0, w=64, h=48, z0=0.0, fy=None):
    c = scenes._identity_cam(w, h, f)
    c.fy = f if fy is None else fy
    c.t = np.array([0.0, 0.0, z0], np.float32)
    return c


def _one(mean, scales=(0.05, 0.02, 0.03), quat=(1.0, 0.0, 0.0, 0.0), op=0.5):
    return SimpleNamespace(means=np.array([mean], np.float64), scales=np.array([scales], np.float64),
                           quats=np.array([quat], np.float64), opacity=np.array([op]),
                           sh=np.zeros((1, 1, 3)), sh_degree=0, n=1)


def test_filter_3d_variance_from_the_sampling_rate():
    # one camera: v = s2 (z / f)^2
    v = O.filter_3d([_cam(f=100.0)], [[0.0, 0.0, 2.0]], s2=0.2)
    assert abs(v[0] - 0.2 * (2.0 / 100.0) ** 2) < 1e-18
    # two cameras: the higher sampling rate (the nearer camera) sets the filter
    far = _cam(f=100.0, z0=2.0)                          # the point sits at depth 4 there
    v = O.filter_3d([far, _cam(f=100.0)], [[0.0, 0.0, 2.0]], s2=0.2)
    assert abs(v[0] - 0.2 * (2.0 / 100.0) ** 2) < 1e-18
    # the larger focal length of a non-square camera counts
    v = O.filter_3d([_cam(f=100.0, fy=150.0)], [[0.0, 0.0, 3.0]], s2=0.5)
    assert abs(v[0] - 0.5 * (3.0 / 150.0) ** 2) < 1e-18
    # unseen: behind the camera, in front of the near plane, outside the image
    v = O.filter_3d([_cam()], [[0.0, 0.0, -1.0], [0.0, 0.0, 0.1], [5.0, 0.0, 1.0]], s2=0.2)
    assert np.all(v == 0.0)
    # the image edge itself counts as seen (centre at u = W exactly)
    c = _cam(f=100.0, w=64)
    x = (64 - c.cx) / 100.0 * 2.0
    assert O.filter_3d([c], [[x, 0.0, 2.0]])[0] > 0


def test_3d_filter_projection_closed_form():
    """Axis-aligned Gaussian on the optical axis: the 3D filter adds v to
    each squared scale, Sigma2D = diag(f^2 (s_x^2 + v), f^2 (s_y^2 + v)) / z^2,
    and the opacity factor is prod_k s_k / sqrt(s_k^2 + v)."""
    f, z, v = 100.0, 2.0, 4e-4
    s = np.array([0.05, 0.02, 0.03])
    p = O.project(_cam(f=f), _one([0.0, 0.0, z], scales=tuple(s)), filt3d=np.array([v]), kernel2d=0.3)
    a = f * f * (s[0] ** 2 + v) / z ** 2 + 0.3
    c = f * f * (s[1] ** 2 + v) / z ** 2 + 0.3
    assert np.allclose(p.cov2d[0], [a, 0.0, c], rtol=1e-12, atol=1e-15)
    assert np.allclose(p.conic[0], [1 / a, 0.0, 1 / c], rtol=1e-12, atol=1e-15)
    assert abs(p.opac_scale[0] - np.prod(s / np.sqrt(s * s + v))) < 1e-14


def test_2d_mip_filter_closed_form_and_mass_conservation():
    f, z = 100.0, 2.0
    s = (0.01, 0.004, 0.02)
    p = O.project(_cam(f=f), _one([0.0, 0.0, z], scales=s), kernel2d=0.1, antialias=True)
    a0, c0 = (f * s[0] / z) ** 2, (f * s[1] / z) ** 2
    assert np.allclose(p.conic[0], [1 / (a0 + 0.1), 0.0, 1 / (c0 + 0.1)], rtol=1e-12, atol=1e-15)
    assert abs(p.opac_scale[0] - np.sqrt(a0 * c0 / ((a0 + 0.1) * (c0 + 0.1)))) < 1e-14
    # for any Gaussian, opacity x footprint area is preserved by the filter:
    # (o rho)^2 det(Sigma2D + k I) = o^2 det(Sigma2D)
    sc = scenes.config0_scene(seed=7, n=300)
    pr = O.project(sc.cameras[0], sc.gaussians, kernel2d=0.1, antialias=True)
    vis = pr.visible == 1
    a, b, c = pr.cov2d[vis].T
    det1 = a * c - b * b
    det0 = (a - 0.1) * (c - 0.1) - b * b
    assert np.allclose(pr.opac_scale[vis] ** 2 * det1, det0, rtol=1e-9, atol=1e-18)
    # without antialiasing the factor is 1; kernel 0 with antialiasing is 1 too
    assert np.all(O.project(sc.cameras[0], sc.gaussians, kernel2d=0.1).opac_scale == 1.0)
    p0 = O.project(sc.cameras[0], sc.gaussians, kernel2d=0.0, antialias=True)
    assert np.allclose(p0.opac_scale[p0.visible == 1], 1.0, rtol=0, atol=1e-12)


def test_gradient_oracle_with_mip_filters_matches_finite_differences():
    s = scenes.config0_scene(seed=3, n=800)
    s.bg = np.array([0.2, 0.3, 0.4], np.float32)
    flt = dict(filt3d=O.filter_3d(s.cameras, s.gaussians.means, s2=0.2), kernel2d=0.1, antialias=True)
    assert np.mean(flt["filt3d"] > 0) > 0.9          # the rest project outside the image
    checked, worst = _check(s, n_per_kind=11, seed=4, flt=flt)
    assert checked >= 50
