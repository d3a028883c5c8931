"""Pins of the CPU FP64 oracle against facts fixed by the paper's equations and
by mathematics (no GPU).  Each test names the equation or passage it pins and
is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign
or index, a transposed operand) fails it.

Eq. 1  Gaussian;  Sec. 3.1  Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T;
Eq. 2  front-to-back alpha blending;  Sec. 3.4  mesh cut-off D_gs < D_m and
I_h = I_gs + T * I_m (I_bg without a triangle);  Sec. 3.1 "Textured mesh"
barycentric UV interpolation + texture lookup.
"""
import math
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_06988_b300 import scenes

C0 = 0.5 / math.sqrt(math.pi)          # Y_0^0 = 1 / (2 sqrt(pi))


def _f32(x):
    return float(np.float32(x))


# ---------------------------------------------------------------- blending --

def test_lone_gaussian_peaks_at_its_opacity():
    """Eq. 2 with one Gaussian centred on a pixel: G' = 1 there, so
    sigma = o, I = o c + (1 - o) I_bg and T = 1 - o."""
    s = scenes.micro_lone_gaussian(px=10, py=12, opacity=0.6)
    s.bg = np.array([0.1, 0.2, 0.3], np.float32)
    r = O.render(s)
    q = 12 * 32 + 10
    o = _f32(0.6)
    c = 0.5 + C0 * s.gaussians.sh[0, 0].astype(np.float64)
    bg = s.bg.astype(np.float64)
    np.testing.assert_allclose(r.out.rgb[:, q], o * c + (1 - o) * bg, rtol=0, atol=1e-12)
    assert abs(r.out.T[q] - (1 - o)) < 1e-12
    assert r.out.n_contrib[q] == 1


def test_alpha_clamp_099():
    """alpha = min(0.99, o G): an opaque Gaussian leaves T = 0.01."""
    s = scenes.micro_lone_gaussian(opacity=1.0)
    r = O.render(s)
    q = 12 * 32 + 10
    assert abs(r.out.T[q] - 0.01) < 1e-12
    c = 0.5 + C0 * s.gaussians.sh[0, 0].astype(np.float64)
    np.testing.assert_allclose(r.out.rgb[:, q], 0.99 * c, atol=1e-12)


def test_two_gaussians_front_to_back():
    """Eq. 2 with two Gaussians on one pixel: a1 c1 + (1-a1) a2 c2 + T bg,
    nearer one first; swapping the depths swaps the roles."""
    for z1, z2 in ((2.0, 2.5), (2.5, 2.0)):
        s = scenes.micro_two_gaussians(z1=z1, z2=z2, o1=0.5, o2=0.7)
        s.bg = np.array([0.05, 0.1, 0.15], np.float32)
        r = O.render(s)
        q = 16 * 32 + 16
        a = [_f32(0.5), _f32(0.7)]
        c = [0.5 + C0 * s.gaussians.sh[i, 0].astype(np.float64) for i in range(2)]
        f, b = (0, 1) if z1 < z2 else (1, 0)
        want = a[f] * c[f] + (1 - a[f]) * a[b] * c[b] + (1 - a[f]) * (1 - a[b]) * s.bg
        # each mean projects onto the pixel centre up to FP32 rounding of the mean
        np.testing.assert_allclose(r.out.rgb[:, q], want, atol=1e-9)
        assert r.out.n_contrib[q] == 2


def test_equal_depth_tie_lower_index_first():
    """Equal FP32 depths are blended in index order (stable order)."""
    s = scenes.micro_two_gaussians(z1=2.0, z2=2.0, o1=0.5, o2=0.7)
    r = O.render(s)
    q = 16 * 32 + 16
    a = [_f32(0.5), _f32(0.7)]
    c = [0.5 + C0 * s.gaussians.sh[i, 0].astype(np.float64) for i in range(2)]
    want = a[0] * c[0] + (1 - a[0]) * a[1] * c[1]
    np.testing.assert_allclose(r.out.rgb[:, q], want, atol=1e-9)


def test_weights_plus_transmittance_telescope_to_one():
    """Telescoping of Eq. 2: sum_i w_i + T_final = 1 (white Gaussians, black
    background, no mesh) to FP64 rounding."""
    s = scenes.config0_scene(seed=3)
    s.mesh = None
    g = s.gaussians
    g.sh = np.full_like(g.sh, np.float32(0.5 / C0))   # colour exactly 1 up to FP32 rounding of sh
    r = O.render(s)
    c = 0.5 + C0 * np.float64(np.float32(0.5 / C0))
    total = r.out.rgb[0] / c + r.out.T
    assert np.abs(total - 1.0).max() < 1e-12
    assert r.out.n_contrib.max() > 5


def test_transmittance_stop():
    """Blending stops before T would fall below 1e-4: with many opaque
    Gaussians on one pixel, exactly two blend (0.01^2 = 1e-4 is not < 1e-4,
    0.01^3 is) and T ends at 0.01^2."""
    cam = scenes._identity_cam()
    n = 6
    zs = np.linspace(2.0, 3.0, n)
    means = np.array([[(16.5 - 16) / 32 * z, (16.5 - 16) / 32 * z, z] for z in zs], np.float32)
    g = scenes.Gaussians(means, np.full((n, 3), 0.05, np.float32), np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
                         np.ones(n, np.float32), np.full((n, 1, 3), 0.3, np.float32), 0)
    s = scenes.Scene("stop", 0, g, None, [cam])
    r = O.render(s)
    q = 16 * 32 + 16
    # 0.01 * 0.01 = 1e-4 in FP64 is 1.0000000000000002e-4 >= 1e-4: two blend,
    # the third would give 1e-6 < 1e-4 and stops the pixel
    assert r.out.n_contrib[q] == 2
    assert abs(r.out.T[q] - 0.01 * 0.01) < 1e-15


# ----------------------------------------------------------- hybrid (3.4) --

def test_gaussians_behind_mesh_contribute_exactly_zero():
    """Sec. 3.4: only Gaussians with D_gs < D_m are blended.  Removing every
    Gaussian behind the z=3 quad of the config-0 scene changes no bit of the
    image, T or counts; removing one in front does."""
    s = scenes.config0_scene(seed=0)
    r = O.render(s)
    behind = s.gaussians.means[:, 2] > 3.0 + 0.1
    assert behind.sum() > 300
    s2 = scenes.config0_scene(seed=0)
    s2.gaussians = s.gaussians.subset(~behind)
    r2 = O.render(s2)
    assert np.array_equal(r.out.rgb, r2.out.rgb)
    assert np.array_equal(r.out.T, r2.out.T)
    assert np.array_equal(r.out.n_contrib, r2.out.n_contrib)
    s3 = scenes.config0_scene(seed=0)
    keep = np.ones(s.gaussians.n, bool)
    keep[np.argmax(np.where(~behind, s.gaussians.opacity, 0))] = False
    s3.gaussians = s.gaussians.subset(keep)
    r3 = O.render(s3)
    assert not np.array_equal(r.out.rgb, r3.out.rgb)


def test_mesh_only_scene_returns_its_texture():
    """With no Gaussians, I_h = I_m and T = 1 on covered pixels; I_bg elsewhere."""
    s = scenes.micro_quad_only(tex=np.full((8, 8, 3), [10, 200, 255], np.uint8))
    r = O.render(s)
    assert (r.mesh.tri_id >= 0).all()
    np.testing.assert_allclose(r.out.rgb, np.repeat(np.array([10, 200, 255])[:, None] / 255.0, 32 * 32, 1),
                               atol=1e-15)
    assert np.all(r.out.T == 1.0)
    s.mesh.verts[:, 2] = -1.0   # behind the camera: no triangle, background
    s.bg = np.array([0.25, 0.5, 0.75], np.float32)
    r = O.render(s)
    assert (r.mesh.tri_id < 0).all()
    np.testing.assert_allclose(r.out.rgb, np.repeat(s.bg[:, None].astype(np.float64), 32 * 32, 1), atol=0)


def test_texel_aligned_quad_reproduces_texture():
    """A fronto-parallel quad exactly covering a W x H view with UVs [0,1]
    and a W x H texture puts texel centre (x+1/2)/W on pixel centre x+1/2:
    bilinear weights are (1,0,0,0) and the texture comes back."""
    W = H = 16
    f = 16.0
    z = 2.0
    cam = scenes.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), f, f, W / 2, H / 2, W, H)
    s_ = (W / 2) / f * z
    verts = np.array([[-s_, -s_, z], [s_, -s_, z], [s_, s_, z], [-s_, s_, z]], np.float32)
    uvs = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    tex = np.random.default_rng(7).integers(0, 256, (H, W, 3), dtype=np.uint8)
    mesh = scenes.Mesh(verts, uvs, np.array([[0, 1, 2], [0, 2, 3]], np.int32), tex)
    m = O.mesh_raster(cam, mesh)
    assert (m.tri_id >= 0).all()
    want = (tex.astype(np.float64) / 255.0).reshape(-1, 3).T
    np.testing.assert_allclose(m.rgb, want, atol=1e-12)
    assert np.all(m.depth == np.float32(2.0))


def test_checkerboard_bilinear_closed_form():
    """2x2 texture [[a,b],[c,d]] on the aligned quad: the sample at (u,v) is
    the bilinear blend with weights s' = clamp(2u - 1/2, 0, 1),
    t' = clamp(2v - 1/2, 0, 1)."""
    W = H = 24
    f = 24.0
    z = 2.0
    cam = scenes.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), f, f, W / 2, H / 2, W, H)
    s_ = (W / 2) / f * z
    verts = np.array([[-s_, -s_, z], [s_, -s_, z], [s_, s_, z], [-s_, s_, z]], np.float32)
    uvs = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    tex = np.array([[[255, 0, 40], [0, 255, 80]], [[0, 128, 120], [255, 64, 160]]], np.uint8)
    mesh = scenes.Mesh(verts, uvs, np.array([[0, 1, 2], [0, 2, 3]], np.int32), tex)
    m = O.mesh_raster(cam, mesh)
    x = np.arange(W) + 0.5
    u = np.tile(x / W, H)
    v = np.repeat((np.arange(H) + 0.5) / H, W)
    sp = np.clip(2 * u - 0.5, 0, 1)[None]
    tp = np.clip(2 * v - 0.5, 0, 1)[None]
    t = tex.astype(np.float64) / 255.0
    a, b, c, d = (t[0, 0][:, None], t[0, 1][:, None], t[1, 0][:, None], t[1, 1][:, None])
    want = (1 - sp) * (1 - tp) * a + sp * (1 - tp) * b + (1 - sp) * tp * c + sp * tp * d
    np.testing.assert_allclose(m.rgb, want, atol=1e-12)


def test_shared_edge_top_left_rule_is_watertight():
    """The quad's diagonal runs exactly through pixel centres: the fill rule
    assigns every covered pixel to exactly one of the two triangles."""
    s = scenes.config0_scene()
    cam = s.cameras[0]
    cover = np.zeros(128 * 128, int)
    for fi in range(2):
        m = s.mesh
        one = scenes.Mesh(m.verts, m.uvs, m.faces[fi:fi + 1], m.texture)
        r = O.mesh_raster(cam, one)
        cover += (r.tri_id >= 0)
    assert cover.min() == 1 and cover.max() == 1
    both = O.mesh_raster(cam, s.mesh)
    on_diag = np.array([both.tri_id[y * 128 + y] for y in range(128)])
    assert set(on_diag.tolist()) <= {0, 1}


@pytest.mark.parametrize("scene_fn,npix", [(scenes.config0_scene, None), ("room", 4000)])
def test_mesh_hits_match_independent_ray_cast(scene_fn, npix):
    """tri_id of the fixed-point rasteriser equals the nearest hit of an FP64
    Moller-Trumbore ray cast through the pixel centre, except on pixels whose
    centre lies within 1e-6 (barycentric) of an edge; depth equals the ray's
    view z to 2e-4 relative (snapping vertices to 1/256 px moves the plane
    of a triangle seen at a grazing angle by that much; interpolating z
    instead of 1/z in screen space would be off by ~1e-2 on these faces)."""
    if scene_fn == "room":
        s = scenes.room_scene(11, n_tris=4000, n_gauss=10, resolutions=((320, 240),))
    else:
        s = scene_fn()
    cam = s.cameras[0]
    rng = np.random.default_rng(0)
    pix = None if npix is None else np.sort(rng.choice(cam.n_pixels, npix, replace=False))
    m = O.mesh_raster(cam, s.mesh, pix=pix)
    rc = O.mesh_raycast(cam, s.mesh, pix=pix)
    ok = rc.edge_bary > 1e-6
    assert ok.mean() > 0.95
    assert np.array_equal(m.tri_id[ok], rc.tri_id[ok])
    hit = ok & (m.tri_id >= 0)
    np.testing.assert_allclose(m.depth[hit].astype(np.float64), rc.z[hit], rtol=2e-4)
    assert np.median(np.abs(m.depth[hit] / rc.z[hit] - 1)) < 1e-5


def _snapped_plane_depth(cam, mesh, tri, pix):
    """Independent statement of the mesh depth (Sec. 3.4 D_m): unproject the
    face's snapped vertices (1/256 px) at their FP64 view depths and
    intersect the pixel-centre ray with the plane through them (3D
    geometry, no screen-space interpolation)."""
    c = O.cam_array(cam)                     # the camera as both renderers take it (FP32 values)
    R, t = c[:9].reshape(3, 3), c[9:12]
    fx, fy, cx, cy = c[12:16]
    W = cam.width
    out = np.empty(len(pix))
    for j, (f, q) in enumerate(zip(tri, pix)):
        P = []
        for vi in mesh.faces[f]:
            X, Y, Z = R @ np.asarray(mesh.verts[vi], np.float64) + t
            sx = np.rint(256.0 * (fx * (X / Z) + cx)) / 256.0
            sy = np.rint(256.0 * (fy * (Y / Z) + cy)) / 256.0
            P.append(Z * np.array([(sx - cx) / fx, (sy - cy) / fy, 1.0]))
        nrm = np.cross(P[1] - P[0], P[2] - P[0])
        x, y = q % W + 0.5, q // W + 0.5
        d = np.array([(x - cx) / fx, (y - cy) / fy, 1.0])
        out[j] = nrm @ P[0] / (nrm @ d)          # ray parameter = view z (d_z = 1)
    return out


@pytest.mark.parametrize("which", ["config0", "room"])
def test_mesh_depth_is_the_snapped_face_plane_in_fp64(which):
    """D_m is the view z where the pixel-centre ray meets the plane of the
    snapped face, in FP64, rounded once to FP32 for the stored depth."""
    if which == "room":
        s = scenes.room_scene(11, n_tris=4000, n_gauss=10, resolutions=((320, 240),))
    else:
        s = scenes.config0_scene()
    cam = s.cameras[0]
    rng = np.random.default_rng(3)
    pix = np.sort(rng.choice(cam.n_pixels, 1500, replace=False))
    m = O.mesh_raster(cam, s.mesh, pix=pix)
    hit = m.tri_id >= 0
    assert hit.mean() > 0.3
    want = _snapped_plane_depth(cam, s.mesh, m.tri_id[hit], pix[hit])
    np.testing.assert_allclose(m.depth64[hit], want, rtol=1e-11)
    assert np.array_equal(m.depth[hit], m.depth64[hit].astype(np.float32))
    # the band sizes a few FP32 ulps: between 3 and 1000 u relative here
    rel = m.depth_tol[hit] / m.depth64[hit]
    assert rel.min() >= 3 * 2.0 ** -24 and rel.max() < 1e3 * 2.0 ** -24


def test_config0_has_no_ambiguous_decision():
    """The default config-0 seed puts no decision of the walk, and no
    nearest-face decision, inside its FP32 band: every pixel is checked
    exactly."""
    r = O.render(scenes.config0_scene())
    assert int(r.out.amb.sum()) == 0
    assert int(r.out.n_amb.sum()) == 0
    assert np.isfinite(r.out.margin).any() and r.out.margin.min() >= 1.0


def _one_gaussian_proj(mx, my, var, depth=2.0, colour=(0.9, 0.2, 0.1)):
    return SimpleNamespace(visible=np.array([1], np.int32), depth=np.array([depth], np.float32),
                           mean2d=np.array([[mx, my]]), cov2d=np.array([[var, 0.0, var]]),
                           conic=np.array([[1.0 / var, 0.0, 1.0 / var]]),
                           color=np.array([list(colour)]))


def _cam16():
    return scenes.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 16.0, 16.0, 8.0, 8.0,
                         16, 16)


@pytest.mark.parametrize("rel,ambiguous", [(1e-10, True), (-1e-10, True), (1e-3, False)])
def test_band_flags_the_three_sigma_edge_and_lists_both_outcomes(rel, ambiguous):
    """A Gaussian whose 3-sigma ellipse passes within 1e-10 (relative) of a
    pixel centre makes that pixel ambiguous; its two valid outcomes are the
    background alone and o e^{-d^2/2} of the colour over it (Eq. 2, one
    Gaussian).  1e-3 away the decision is exact."""
    cam = _cam16()
    var = 2.0
    d2 = 9.0 * (1.0 + rel)
    pr = _one_gaussian_proj(4.5 - math.sqrt(d2 * var), 4.5, var)   # pixel (4, 4): centre (4.5, 4.5)
    o = np.array([0.8])
    bg = (0.1, 0.2, 0.3)
    mr = O.empty_mesh_result(1, bg)
    out = O.blend(cam, pr, o, mr, bg=bg, pix=[4 * 16 + 4])
    assert bool(out.amb[0]) == ambiguous
    if not ambiguous:
        assert out.margin[0] >= 1.0
        return
    outs = O.flip_outcomes(cam, pr, o, mr, 0, 4 * 16 + 4, bg=bg)
    assert len(outs) == 2
    a = 0.8 * math.exp(-0.5 * d2)
    by_n = {n: (rgb, T) for rgb, T, n in outs}
    np.testing.assert_allclose(by_n[0][0], bg, atol=1e-15)
    np.testing.assert_allclose(by_n[1][0], a * np.array([0.9, 0.2, 0.1]) + (1 - a) * np.array(bg), atol=1e-15)
    assert abs(by_n[1][1] - (1 - a)) < 1e-15
    # the unflipped walk comes first and is the exact decision
    assert outs[0][2] == (0 if rel > 0 else 1)


def test_band_flags_a_gaussian_at_the_mesh_depth():
    """Sec. 3.4 cut: a Gaussian whose depth equals the mesh depth within the
    mesh pass's FP32 band may be cut or blended; one clearly in front is
    blended, one clearly behind contributes exactly 0."""
    cam = _cam16()
    Im = np.array([[0.5], [0.5], [0.5]])
    for dz, amb in ((0.0, True), (-1e-3, False), (1e-3, False)):
        pr = _one_gaussian_proj(4.5, 4.5, 2.0, depth=np.float32(3.0 + dz))
        mr = SimpleNamespace(tri_id=np.array([0], np.int32), depth=np.array([3.0], np.float32),
                             rgb=Im, depth64=np.array([3.0]), depth_tol=np.array([3.0 * 6 * 2.0 ** -24]),
                             tri2=np.array([-1], np.int32), tri_margin=np.array([np.inf]))
        out = O.blend(cam, pr, np.array([0.8]), mr, pix=[4 * 16 + 4])
        assert bool(out.amb[0]) == amb, dz
        if dz > 0:
            assert out.n_contrib[0] == 0 and out.T[0] == 1.0
        if amb:
            outs = O.flip_outcomes(cam, pr, np.array([0.8]), mr, 0, 4 * 16 + 4)
            assert sorted(n for _, _, n in outs) == [0, 1]
        # the same Gaussian 5 sigma away from the pixel: cut or not, it adds
        # nothing there, so its cut is not a decision of that pixel
        far = _one_gaussian_proj(4.5 + 5 * math.sqrt(2.0), 4.5, 2.0, depth=np.float32(3.0 + dz))
        out = O.blend(cam, far, np.array([0.8]), mr, pix=[4 * 16 + 4])
        assert not out.amb[0] and out.n_contrib[0] == 0 and out.T[0] == 1.0


def _poison(g, rng, k=12):
    """Copy of g with k Gaussians' parameters made non-finite (NaN or +-Inf
    in the mean, scale, quaternion, opacity or SH) or the quaternion zero."""
    import copy
    h = copy.deepcopy(g)
    idx = rng.choice(g.n, k, replace=False)
    kinds = ["mean", "scale", "quat", "opacity", "sh", "zeroquat"]
    for j, i in enumerate(idx):
        bad = [np.nan, np.inf, -np.inf][j % 3]
        kind = kinds[j % len(kinds)]
        if kind == "mean":
            h.means[i, j % 3] = bad
        elif kind == "scale":
            h.scales[i, j % 3] = bad
        elif kind == "quat":
            h.quats[i, j % 4] = bad
        elif kind == "opacity":
            h.opacity[i] = bad
        elif kind == "sh":
            h.sh[i, 0, j % 3] = bad
        else:
            h.quats[i] = 0.0
    return h, np.sort(idx)


def test_non_finite_gaussians_are_culled():
    """Reading: a Gaussian with a non-finite parameter (or a zero
    quaternion) takes no part in the render -- the image, T and counts are
    bit-identical to the render without it."""
    s = scenes.config0_scene()
    bad_g, idx = _poison(s.gaussians, np.random.default_rng(5))
    keep = np.setdiff1d(np.arange(s.gaussians.n), idx)
    a = O.render(s, gaussians=bad_g)
    assert not a.proj.visible[idx].any()
    b = O.render(s, gaussians=s.gaussians.subset(keep))
    for k in ("rgb", "T", "n_contrib"):
        assert np.array_equal(getattr(a.out, k), getattr(b.out, k)), k


# ------------------------------------------------------------ projection --

def test_projected_covariance_closed_form():
    """Sec. 3.1 Sigma' = J W Sigma W^T J^T (+0.3 px^2 dilation): an
    axis-aligned Gaussian on the optical axis at depth z projects to
    diag(fx^2 sx^2 / z^2, fy^2 sy^2 / z^2) + 0.3 at the principal point;
    a 90-degree turn about z swaps the two axes."""
    cam = scenes.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 100.0, 120.0, 50.0, 40.0, 100, 80)
    sx, sy, sz, z = 0.02, 0.05, 0.03, 2.5
    g = SimpleNamespace(means=np.array([[0, 0, z]]), scales=np.array([[sx, sy, sz]]),
                        quats=np.array([[1.0, 0, 0, 0]]), sh=np.zeros((1, 1, 3)), sh_degree=0)
    p = O.project(cam, g)
    want = [100 ** 2 * sx ** 2 / z ** 2 + 0.3, 0.0, 120 ** 2 * sy ** 2 / z ** 2 + 0.3]
    np.testing.assert_allclose(p.cov2d[0], want, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(p.mean2d[0], [50.0, 40.0], atol=1e-13)
    a, b, c = want
    det = a * c - b * b
    np.testing.assert_allclose(p.conic[0], [c / det, -b / det, a / det], rtol=1e-13)
    h = math.sqrt(0.5)
    g.quats = np.array([[h, 0, 0, h]])          # 90 degrees about z: x <-> y
    p = O.project(cam, g)
    want = [100 ** 2 * sy ** 2 / z ** 2 + 0.3, 0.0, 120 ** 2 * sx ** 2 / z ** 2 + 0.3]
    np.testing.assert_allclose(p.cov2d[0], want, rtol=1e-12, atol=1e-12)
    g.quats = np.array([[2.0, 0, 0, 0]])        # quaternions are normalised
    p = O.project(cam, g)
    np.testing.assert_allclose(p.cov2d[0][[0, 2]], [100 ** 2 * sx ** 2 / z ** 2 + 0.3,
                                                    120 ** 2 * sy ** 2 / z ** 2 + 0.3], rtol=1e-13)


def test_projection_offaxis_first_order():
    """Off axis, J's third column adds -fx x/z^2 Sigma_zz-type terms: a
    needle along the optical axis seen off-centre projects to a segment of
    length fx * x * L / z^2 (first order in L), checked by projecting the
    needle's end points."""
    cam = scenes.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 200.0, 200.0, 100.0, 100.0, 200, 200)
    x, z, L = 0.3, 2.0, 1e-3
    g = SimpleNamespace(means=np.array([[x, 0, z]]), scales=np.array([[1e-9, 1e-9, L]]),
                        quats=np.array([[1.0, 0, 0, 0]]), sh=np.zeros((1, 1, 3)), sh_degree=0)
    p = O.project(cam, g)
    # Sigma'_xx - 0.3 = (d u / d z)^2 L^2 with u = fx x / z
    dudz = -200.0 * x / z ** 2
    np.testing.assert_allclose(p.cov2d[0, 0] - 0.3, dudz ** 2 * L ** 2, rtol=1e-9)
    np.testing.assert_allclose(p.cov2d[0, 2] - 0.3, 0.0, atol=1e-12)


def test_near_plane_culls():
    cam = scenes._identity_cam()
    g = SimpleNamespace(means=np.array([[0, 0, 0.19], [0, 0, 0.21], [0, 0, -1.0]]),
                        scales=np.full((3, 3), 0.01), quats=np.tile([1.0, 0, 0, 0], (3, 1)),
                        sh=np.zeros((3, 1, 3)), sh_degree=0)
    p = O.project(cam, g)
    assert p.visible.tolist() == [0, 1, 0]


def test_depth_key_is_rounded_fp64_fma_chain():
    """The depth key is fp32(fma(R20,x,fma(R21,y,fma(R22,z,t2)))): reproduce it
    with exact rational arithmetic of FP32 inputs and a single FP32 rounding
    (the FMA chain in FP64 is exact for these short-mantissa inputs)."""
    from fractions import Fraction
    s = scenes.room_scene(5, n_tris=2000, n_gauss=500, resolutions=((64, 48),))
    cam = s.cameras[0]
    p = O.project(cam, s.gaussians)
    R, t = cam.R.astype(np.float32), cam.t.astype(np.float32)
    for i in range(0, 500, 37):
        m = s.gaussians.means[i]
        exact = sum(Fraction(float(R[2, k])) * Fraction(float(m[k])) for k in range(3)) + Fraction(float(t[2]))
        # all partial sums fit in 53 bits here, so the FP64 chain is exact
        assert np.float32(float(exact)) == p.depth[i]


# --------------------------------------------------------------------- SH --

def test_sh_basis_orthonormal_by_quadrature():
    """The real SH basis used for colour is orthonormal on the sphere:
    Gauss-Legendre in cos(theta) x uniform phi, exact for degree <= 6 products."""
    nt, nphi = 12, 16
    xs, ws = np.polynomial.legendre.leggauss(nt)
    phis = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    G = np.zeros((16, 16))
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = O.sh_basis(3, [st * math.cos(ph), st * math.sin(ph), ct])
            G += w * (2 * np.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_known_values():
    d = np.array([0.36, -0.48, 0.8])
    Y = O.sh_basis(3, d)
    assert abs(Y[0] - 0.5 / math.sqrt(math.pi)) < 1e-15
    k1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[1:4], [-k1 * d[1], k1 * d[2], -k1 * d[0]], atol=1e-15)
    # l=2, m=0: sqrt(5/4pi) (3z^2-1)/2
    assert abs(Y[6] - math.sqrt(5 / (4 * math.pi)) * (3 * d[2] ** 2 - 1) / 2) < 1e-14
    # l=3, m=3: sqrt(35/(32 pi)) * (-(x^3 - 3 x y^2))  (Condon-Shortley phase)
    assert abs(Y[15] - (-math.sqrt(35 / (32 * math.pi)) * (d[0] ** 3 - 3 * d[0] * d[1] ** 2))) < 1e-14


def test_degree0_colour_is_view_independent():
    s = scenes.config0_scene()
    g = s.gaussians
    p = O.project(s.cameras[0], g)
    want = np.maximum(0.0, 0.5 + C0 * g.sh[:, 0, :].astype(np.float64))
    np.testing.assert_allclose(p.color, want, atol=1e-15)


# ------------------------------------------------------ prefilter identity --

def test_grid_prefilter_identical_to_brute_force():
    s = scenes.config0_scene(seed=1)
    a = O.render(s)
    b = O.render(s, mode="grid")
    for k in ("rgb", "T", "n_contrib", "fp", "n_amb", "evaluated"):
        assert np.array_equal(getattr(a.out, k), getattr(b.out, k)), k


def test_grid_prefilter_identical_on_room_crop():
    s = scenes.room_scene(7, n_tris=3000, n_gauss=20000, resolutions=((160, 120),))
    a = O.render(s)
    b = O.render(s, mode="grid")
    for k in ("rgb", "T", "n_contrib", "fp"):
        assert np.array_equal(getattr(a.out, k), getattr(b.out, k)), k


def test_oracle_matches_committed_digest():
    """Regression digest written by tests/golden/make_golden.py (oracle only)."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    try:
        import make_golden
    finally:
        sys.path.pop(0)
    want = json.load(open(os.path.join(here, "config0_oracle_digest.json")))
    got = make_golden.digest()
    for k, v in want.items():
        if isinstance(v, float):
            assert abs(got[k] - v) <= 1e-9 * max(1.0, abs(v)), k
        elif isinstance(v, list) and v and isinstance(v[0], float):
            np.testing.assert_allclose(got[k], v, rtol=1e-12, atol=1e-12)
        else:
            assert got[k] == v, k
