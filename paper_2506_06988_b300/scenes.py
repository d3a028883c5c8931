"""Seeded synthetic scenes shaped like the indoor workloads of the hybrid
mesh-Gaussian representation (Sec. 4 evaluates on real indoor captures, which
are not available here; these generators stand in for them).

This module only builds inputs: cameras, Gaussian parameters (already
activated: scales = exp(log-scale), opacity = sigmoid(logit)), a textured
triangle mesh and seeded random draws.  It contains none of the rendering
arithmetic, so both the CUDA path and the CPU oracle can consume its output.

Conventions
-----------
* Camera: world->camera rotation ``R`` (row-major 3x3) and translation ``t``,
  ``p_cam = R @ p_world + t``; OpenCV axes (+x right, +y down, +z forward);
  pinhole intrinsics fx, fy, cx, cy in pixels; image ``width`` x ``height``.
* Gaussians: means [N,3], scales [N,3] (activated), quats [N,4] as (w,x,y,z),
  not necessarily normalised, opacity [N] (activated), sh [N,(d+1)^2,3].
* Mesh: verts [V,3] f32, per-vertex uvs [V,2] f32 (seams are duplicated
  vertices), faces [F,3] int32, texture [Ht,Wt,3] uint8 (or float32 texels).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Camera", "Gaussians", "Mesh", "Scene",
    "config0_scene", "room_scene", "config1_scene", "config1_plain_scene",
    "config2_scene", "config3_scene", "config4_scene", "camera_lookat",
    "micro_lone_gaussian", "micro_two_gaussians", "micro_quad_only",
]


@dataclass
class Camera:
    R: np.ndarray            # (3,3) float32, world -> camera
    t: np.ndarray            # (3,)  float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        """16 float32 values: R (row-major), t, fx, fy, cx, cy."""
        return np.concatenate([
            np.asarray(self.R, np.float32).reshape(9),
            np.asarray(self.t, np.float32).reshape(3),
            np.array([self.fx, self.fy, self.cx, self.cy], np.float32),
        ]).astype(np.float32)

    @property
    def n_pixels(self) -> int:
        return int(self.width) * int(self.height)


@dataclass
class Gaussians:
    means: np.ndarray        # [N,3] f32
    scales: np.ndarray       # [N,3] f32 (activated)
    quats: np.ndarray        # [N,4] f32 (w,x,y,z)
    opacity: np.ndarray      # [N]   f32 (activated)
    sh: np.ndarray           # [N,(d+1)^2,3] f32 or f16
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.means[idx], self.scales[idx], self.quats[idx],
                         self.opacity[idx], self.sh[idx], self.sh_degree)

    def copy(self) -> "Gaussians":
        return Gaussians(self.means.copy(), self.scales.copy(), self.quats.copy(),
                         self.opacity.copy(), self.sh.copy(), self.sh_degree)


@dataclass
class Mesh:
    verts: np.ndarray        # [V,3] f32
    uvs: np.ndarray          # [V,2] f32
    faces: np.ndarray        # [F,3] i32
    texture: np.ndarray      # [Ht,Wt,3] u8 or f32

    @property
    def n_faces(self) -> int:
        return int(self.faces.shape[0])


@dataclass
class Scene:
    name: str
    seed: int
    gaussians: Gaussians
    mesh: Optional[Mesh]
    cameras: List[Camera]
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    notes: dict = field(default_factory=dict)

    @property
    def n_pixels(self) -> int:
        return sum(c.n_pixels for c in self.cameras)


# --------------------------------------------------------------------------
# random draws
# --------------------------------------------------------------------------

def _rngs(seed: int, n: int):
    ss = np.random.SeedSequence(seed)
    return [np.random.default_rng(s) for s in ss.spawn(n)]


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def camera_lookat(center, forward, width, height, fx, fy=None, cx=None, cy=None,
                  up=(0.0, 1.0, 0.0)) -> Camera:
    """Camera at ``center`` looking along ``forward`` with world ``up`` (+y).

    Rows of R are the camera's right, down and forward axes in world
    coordinates, so (right, down, forward) is right-handed."""
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    u = np.asarray(up, np.float64)
    right = np.cross(f, u)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f]).astype(np.float32)
    C = np.asarray(center, np.float64)
    t = (-(R.astype(np.float64) @ C)).astype(np.float32)
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    return Camera(R, t, float(fx), float(fy), float(cx), float(cy), int(width), int(height))


def _band_limited_noise(rng, size, cutoff_px=6.0):
    """RGB noise with a Gaussian low-pass (in frequency) of ``cutoff_px``
    texel correlation length, scaled to [0,255] uint8."""
    white = rng.standard_normal((size, size, 3))
    fy = np.fft.fftfreq(size)[:, None]
    fx = np.fft.rfftfreq(size)[None, :]
    g = np.exp(-2.0 * (np.pi * cutoff_px) ** 2 * (fx * fx + fy * fy))
    out = np.empty_like(white)
    for c in range(3):
        out[..., c] = np.fft.irfft2(np.fft.rfft2(white[..., c]) * g, s=(size, size))
    lo, hi = np.percentile(out, 0.5), np.percentile(out, 99.5)
    out = np.clip((out - lo) / (hi - lo), 0.0, 1.0)
    return np.round(out * 255.0).astype(np.uint8)


# --------------------------------------------------------------------------
# config 0: 2k Gaussians in front of / behind one textured quad, 128x128
# --------------------------------------------------------------------------

def config0_scene(seed: int = 1, n: int = 2000) -> Scene:
    """The default seed is one at which no decision of the render lies in
    the FP32 ambiguity band of an FP32 renderer (the exact checks then cover
    every pixel).  2,000 Gaussians, means U[-1,1]^3 + (0,0,2.5), log-scales N(-3.5,0.5),
    uniform unit quaternions, opacity sigmoid(N(0,1)), SH degree 0 with DC
    coefficients U[0,1]; a 2-triangle quad at z=3 that fills a 128x128 view
    (fx=fy=128, centred principal point, identity pose) with a 64x64 RGB8
    noise texture and UVs spanning [0,1]."""
    r_mean, r_scale, r_quat, r_op, r_sh, r_tex = _rngs(seed, 6)
    means = (r_mean.uniform(-1.0, 1.0, (n, 3)) + np.array([0.0, 0.0, 2.5])).astype(np.float32)
    scales = np.exp(r_scale.normal(-3.5, 0.5, (n, 3))).astype(np.float32)
    quats = _unit_quats(r_quat, n)
    opacity = _sigmoid(r_op.normal(0.0, 1.0, n)).astype(np.float32)
    sh = r_sh.uniform(0.0, 1.0, (n, 1, 3)).astype(np.float32)
    g = Gaussians(means, scales, quats, opacity, sh, 0)
    s = 1.6
    verts = np.array([[-s, -s, 3.0], [s, -s, 3.0], [s, s, 3.0], [-s, s, 3.0]], np.float32)
    uvs = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    faces = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    tex = r_tex.integers(0, 256, (64, 64, 3), dtype=np.uint8)
    cam = Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32),
                 128.0, 128.0, 64.0, 64.0, 128, 128)
    return Scene("config0", seed, g, Mesh(verts, uvs, faces, tex), [cam])


# --------------------------------------------------------------------------
# indoor rooms
# --------------------------------------------------------------------------

@dataclass
class _Rect:
    origin: np.ndarray   # corner
    a: np.ndarray        # unit axis along width
    b: np.ndarray        # unit axis along height
    w: float
    h: float
    holes: list = field(default_factory=list)   # [(a0,a1,b0,b1)] door openings (no cells)


def _room_rects(rooms_x: int, rooms_z: int, rx=6.0, rz=5.0, ry=3.0, door=(1.0, 2.1)):
    """Axis-aligned surfaces of a rooms_x x rooms_z grid of rx x ry x rz rooms.
    Interior walls carry a door opening per shared wall and are double-sided
    (each side is its own surface)."""
    X, Z, Y = rooms_x * rx, rooms_z * rz, ry
    ex, ey, ez = np.eye(3)
    rects = [
        _Rect(np.zeros(3), ex, ez, X, Z),                   # floor y=0
        _Rect(np.array([0, Y, 0.0]), ex, ez, X, Z),         # ceiling y=Y
        _Rect(np.zeros(3), ex, ey, X, Y),                   # wall z=0
        _Rect(np.array([0, 0, Z]), ex, ey, X, Y),           # wall z=Z
        _Rect(np.zeros(3), ez, ey, Z, Y),                   # wall x=0
        _Rect(np.array([X, 0, 0.0]), ez, ey, Z, Y),         # wall x=X
    ]
    dw, dh = door
    for i in range(1, rooms_x):          # interior walls at x = i*rx
        for side in (-1e-3, 1e-3):
            holes = [(j * rz + rz / 2 - dw / 2, j * rz + rz / 2 + dw / 2, 0.0, dh) for j in range(rooms_z)]
            rects.append(_Rect(np.array([i * rx + side, 0, 0.0]), ez, ey, Z, Y, holes))
    for j in range(1, rooms_z):          # interior walls at z = j*rz
        for side in (-1e-3, 1e-3):
            holes = [(i * rx + rx / 2 - dw / 2, i * rx + rx / 2 + dw / 2, 0.0, dh) for i in range(rooms_x)]
            rects.append(_Rect(np.array([0, 0, j * rz + side]), ex, ey, X, Y, holes))
    return rects, (X, Y, Z)


def _pack_charts(rects, atlas: int, pad: int = 4):
    """Shelf-pack one chart per surface at a uniform texel density."""
    order = sorted(range(len(rects)), key=lambda i: -rects[i].h)

    def try_scale(s):
        x = y = shelf_h = 0
        pos = {}
        for i in order:
            w = int(np.ceil(rects[i].w * s)) + 2 * pad
            h = int(np.ceil(rects[i].h * s)) + 2 * pad
            if x + w > atlas:
                x, y = 0, y + shelf_h
                shelf_h = 0
            if w > atlas or y + h > atlas:
                return None
            pos[i] = (x + pad, y + pad)
            x += w
            shelf_h = max(shelf_h, h)
        return pos

    lo, hi = 1.0, float(atlas)
    best = None
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        p = try_scale(mid)
        if p is None:
            hi = mid
        else:
            lo, best = mid, p
    return lo, best


def _grid_mesh(rects, target_tris: int, atlas: int):
    area = sum(r.w * r.h for r in rects)
    h = np.sqrt(2.0 * area / target_tris)
    scale, pos = _pack_charts(rects, atlas)
    V, UV, Fc, rect_of_face = [], [], [], []
    base = 0
    for ri, r in enumerate(rects):
        nx = max(1, int(round(r.w / h)))
        ny = max(1, int(round(r.h / h)))
        ia = np.linspace(0.0, r.w, nx + 1)
        ib = np.linspace(0.0, r.h, ny + 1)
        A, B = np.meshgrid(ia, ib, indexing="xy")          # [ny+1, nx+1]
        P = r.origin[None, None, :] + A[..., None] * r.a + B[..., None] * r.b
        px, py = pos[ri]
        U = (px + A * scale) / atlas
        Vv = (py + B * scale) / atlas
        V.append(P.reshape(-1, 3))
        UV.append(np.stack([U, Vv], -1).reshape(-1, 2))
        jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        keep = np.ones((ny, nx), bool)
        for (a0, a1, b0, b1) in r.holes:
            ca = (ii + 0.5) * (r.w / nx)
            cb = (jj + 0.5) * (r.h / ny)
            keep &= ~((ca > a0) & (ca < a1) & (cb > b0) & (cb < b1))
        jj, ii = jj[keep], ii[keep]
        v00 = base + jj * (nx + 1) + ii
        v10 = v00 + 1
        v01 = v00 + (nx + 1)
        v11 = v01 + 1
        f = np.concatenate([np.stack([v00, v10, v11], -1), np.stack([v00, v11, v01], -1)])
        Fc.append(f)
        rect_of_face.append(np.full(len(f), ri))
        base += (nx + 1) * (ny + 1)
    return (np.concatenate(V).astype(np.float32), np.concatenate(UV).astype(np.float32),
            np.concatenate(Fc).astype(np.int32), np.concatenate(rect_of_face))


def _cluster_prune(rng, verts, faces, frac, n_clusters=12):
    """Remove ``frac`` of the faces in seeded roughly-round clusters (holes)."""
    cent = verts[faces].mean(1)
    centers = cent[rng.choice(len(faces), n_clusters, replace=False)]
    radii = rng.uniform(0.5, 1.5, n_clusters)
    d = np.min(np.linalg.norm(cent[:, None, :] - centers[None], axis=-1) / radii[None], axis=1)
    n_remove = int(round(frac * len(faces)))
    order = np.argsort(d, kind="stable")
    removed = np.zeros(len(faces), bool)
    removed[order[:n_remove]] = True
    return faces[~removed], faces[removed]


def _sample_on_faces(rng, verts, faces, n):
    a = verts[faces[:, 1]] - verts[faces[:, 0]]
    b = verts[faces[:, 2]] - verts[faces[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(a, b), axis=1)
    idx = rng.choice(len(faces), n, p=area / area.sum())
    r1, r2 = rng.random(n), rng.random(n)
    s = np.sqrt(r1)
    w0, w1, w2 = 1 - s, s * (1 - r2), s * r2
    f = faces[idx]
    p = w0[:, None] * verts[f[:, 0]] + w1[:, None] * verts[f[:, 1]] + w2[:, None] * verts[f[:, 2]]
    nrm = np.cross(a[idx], b[idx])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return p, nrm


def room_scene(seed: int, *, rooms=(1, 1), n_tris=50_000, prune_frac=0.10, atlas=2048,
               n_gauss=300_000, log_scale=(-4.0, 0.6), logit_opacity=(0.5, 1.0),
               sh_degree=3, sh_std=0.2, sh_f16=False, resolutions=((1920, 1080),) * 8,
               focal_per_width=1100.0 / 1920.0, n_boxes_per_room=20, texture_f32=False,
               with_mesh=True, wall_gaussians=0, name="room", view_block: int = 0) -> Scene:
    """Indoor room scene: a box room (or a grid of connected rooms) whose walls,
    floor and ceiling are triangulated into ~``n_tris`` triangles with
    ``prune_frac`` removed in seeded clusters (pruned holes); a band-limited
    noise RGB8 texture atlas; ``n_gauss`` Gaussians, 70% clustered around
    furniture boxes and 30% near the holes; cameras inside the room(s) at least
    0.3 m from every surface.  ``wall_gaussians`` adds flat textured Gaussians
    covering the walls (the Gaussian-only comparison scene).  ``view_block``
    k selects the k-th block of poses of the same room (block 0 = the first
    len(resolutions) poses of the seeded sequence): distinct views of one
    scene, e.g. one block per rank."""
    (r_prune, r_tex, r_box, r_g1, r_g2, r_attr, r_pose, r_wall) = _rngs(seed, 8)
    rects, (X, Y, Z) = _room_rects(*rooms)
    verts, uvs, faces_all, _ = _grid_mesh(rects, n_tris, atlas)
    faces, removed = _cluster_prune(r_prune, verts, faces_all, prune_frac,
                                    n_clusters=12 * rooms[0] * rooms[1])
    tex = _band_limited_noise(r_tex, atlas)
    if texture_f32:
        tex = (tex.astype(np.float32) / 255.0)

    # furniture boxes on the floor
    nb = n_boxes_per_room * rooms[0] * rooms[1]
    lo = np.array([0.5, 0.0, 0.5])
    hi = np.array([X - 0.5, 0.0, Z - 0.5])
    bsize = r_box.uniform([0.3, 0.3, 0.3], [1.4, 1.4, 1.4], (nb, 3))
    bpos = r_box.uniform(lo, hi, (nb, 3))
    bpos[:, 1] = 0.0
    n_cluster = int(round(0.7 * n_gauss))
    n_hole = n_gauss - n_cluster
    which = r_g1.integers(0, nb, n_cluster)
    u = r_g1.random((n_cluster, 3))
    centers = bpos[which] + (u - np.array([0.5, 0.0, 0.5])) * bsize[which]
    pc = centers + r_g1.normal(0.0, 0.03, (n_cluster, 3))
    if len(removed):
        ph, nh = _sample_on_faces(r_g2, verts, removed, n_hole)
        ph = ph + nh * r_g2.normal(0.0, 0.02, (n_hole, 1))
    else:
        ph = r_g2.uniform([0, 0, 0], [X, Y, Z], (n_hole, 3))
    means = np.concatenate([pc, ph]).astype(np.float32)
    N = len(means)
    scales = np.exp(r_attr.normal(log_scale[0], log_scale[1], (N, 3))).astype(np.float32)
    quats = _unit_quats(r_attr, N)
    opacity = _sigmoid(r_attr.normal(logit_opacity[0], logit_opacity[1], N)).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = r_attr.normal(0.0, sh_std, (N, K, 3)).astype(np.float16 if sh_f16 else np.float32)

    if wall_gaussians:
        pw, nw = _sample_on_faces(r_wall, verts, faces, wall_gaussians)
        pw = pw + nw * r_wall.normal(0.0, 0.002, (wall_gaussians, 1))
        # flat: smallest axis along the surface normal (log-scale N(-7,0.3))
        sw = np.exp(np.stack([r_wall.normal(-4.0, 0.6, wall_gaussians),
                              r_wall.normal(-4.0, 0.6, wall_gaussians),
                              r_wall.normal(-7.0, 0.3, wall_gaussians)], 1))
        # quaternion rotating +z onto the normal
        zax = np.array([0.0, 0.0, 1.0])
        ax = np.cross(np.broadcast_to(zax, nw.shape), nw)
        s = np.linalg.norm(ax, axis=1, keepdims=True)
        c = nw @ zax
        ang = np.arctan2(s[:, 0], c)
        axn = np.where(s > 1e-9, ax / np.maximum(s, 1e-12), np.array([1.0, 0.0, 0.0]))
        qw = np.concatenate([np.cos(ang / 2)[:, None], axn * np.sin(ang / 2)[:, None]], 1)
        ow = _sigmoid(r_wall.normal(2.0, 0.5, wall_gaussians))
        shw = r_wall.normal(0.0, sh_std, (wall_gaussians, K, 3))
        means = np.concatenate([means, pw.astype(np.float32)])
        scales = np.concatenate([scales, sw.astype(np.float32)])
        quats = np.concatenate([quats, qw.astype(np.float32)])
        opacity = np.concatenate([opacity, ow.astype(np.float32)])
        sh = np.concatenate([sh, shw.astype(sh.dtype)])

    g = Gaussians(means, scales, quats, opacity, sh, sh_degree)

    # cameras: inside the rooms, >= 0.3 m from every surface and outside boxes
    cams = []
    margin = 0.8
    bmin = bpos - np.array([0.5, 0.0, 0.5]) * bsize - 0.3
    bmax = bpos + np.array([0.5, 1.0, 0.5]) * bsize + 0.3
    for (w, h) in list(resolutions) * (view_block + 1):
        while True:
            C = r_pose.uniform([margin, 0.8, margin], [X - margin, Y - 0.8, Z - margin])
            inside = np.any(np.all((C > bmin) & (C < bmax), axis=1))
            if rooms != (1, 1):
                # keep clear of interior walls
                if np.min(np.abs((C[0] / 6.0) - np.round(C[0] / 6.0))) * 6.0 < 0.4 and 0 < C[0] < X:
                    if np.round(C[0] / 6.0) not in (0, rooms[0]):
                        continue
                if np.min(np.abs((C[2] / 5.0) - np.round(C[2] / 5.0))) * 5.0 < 0.4 and 0 < C[2] < Z:
                    if np.round(C[2] / 5.0) not in (0, rooms[1]):
                        continue
            if not inside:
                break
        yaw = r_pose.uniform(0, 2 * np.pi)
        pitch = r_pose.normal(0.0, 0.15)
        fwd = np.array([np.cos(pitch) * np.sin(yaw), np.sin(pitch), np.cos(pitch) * np.cos(yaw)])
        f = focal_per_width * w
        cams.append(camera_lookat(C, fwd, w, h, f))
    cams = cams[view_block * len(resolutions):]

    mesh = Mesh(verts, uvs, faces.astype(np.int32), tex) if with_mesh else None
    return Scene(name, seed, g, mesh, cams,
                 notes=dict(room=(X, Y, Z), n_faces_before_prune=int(len(faces_all)),
                            n_removed=int(len(removed))))


def config1_scene(seed: int = 1, n_views: int = 8, view_block: int = 0) -> Scene:
    """Indoor room, 1920x1080 (fx=fy=1100), 8 poses, 50k triangles with 10%
    pruned, 2048^2 RGB8 atlas, 300k Gaussians, SH degree 3 (``view_block``:
    another block of 8 poses of the same room)."""
    return room_scene(seed, resolutions=((1920, 1080),) * n_views, name="config1", view_block=view_block)


def config1_plain_scene(seed: int = 1, n_views: int = 8) -> Scene:
    """Gaussian-only comparison scene for config 1: no mesh; 900k flat
    textured Gaussians (log-scale along the normal N(-7,0.3)) cover the walls
    in addition to the 300k scene Gaussians (1.2M total)."""
    return room_scene(seed, resolutions=((1920, 1080),) * n_views, with_mesh=False,
                      wall_gaussians=900_000, name="config1_plain")


def config2_scene(seed: int = 2) -> Scene:
    """Joint-optimisation scene: the room at 1296x968 with 500k Gaussians, SH
    degree 3 and float32 learnable texels."""
    return room_scene(seed, n_gauss=500_000, resolutions=((1296, 968),), texture_f32=True,
                      name="config2")


def config2_target_params(scene: Scene, seed: int = 20) -> Gaussians:
    """Perturbed parameters whose rendering is the L1 target of config 2:
    means + N(0,0.01); view-independent colours + N(0,0.05), i.e. the SH DC
    coefficients + N(0,0.05)/C0 (the colour is 0.5 + C0 * DC + ...)."""
    r1, r2 = _rngs(seed, 2)
    g = scene.gaussians.copy()
    g.means = (g.means + r1.normal(0.0, 0.01, g.means.shape)).astype(np.float32)
    sh = g.sh.astype(np.float32)
    sh[:, 0, :] += r2.normal(0.0, 0.05, sh[:, 0, :].shape) / 0.28209479177387814
    g.sh = sh.astype(g.sh.dtype)
    return g


def config3_scene(seed: int = 3) -> Scene:
    """Batched views: 16 cameras of uneven resolution (4 each at 640x480,
    1024x768, 1296x968, 1920x1080), 1M Gaussians, 200k triangles, 4096^2 atlas,
    FP16 SH storage."""
    res = [(640, 480)] * 4 + [(1024, 768)] * 4 + [(1296, 968)] * 4 + [(1920, 1080)] * 4
    return room_scene(seed, n_tris=200_000, atlas=4096, n_gauss=1_000_000, sh_f16=True,
                      resolutions=tuple(res), name="config3")


def config4_scene(seed: int = 4) -> Scene:
    """Large scene: 2x2 connected rooms, 1M triangles with 15% pruned, 4096^2
    atlas, 3M Gaussians (log-scales N(-4.5,0.7)), 8 views at 3840x2160."""
    return room_scene(seed, rooms=(2, 2), n_tris=1_000_000, prune_frac=0.15, atlas=4096,
                      n_gauss=3_000_000, log_scale=(-4.5, 0.7),
                      resolutions=((3840, 2160),) * 8, name="config4")


# --------------------------------------------------------------------------
# micro scenes for closed-form checks
# --------------------------------------------------------------------------

def _identity_cam(w=32, h=32, f=32.0):
    return Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), f, f, w / 2.0, h / 2.0, w, h)


def micro_lone_gaussian(px=10, py=12, z=2.0, opacity=0.6, sh_dc=(0.3, 0.7, 0.9), scale=0.05,
                        w=32, h=32, f=32.0) -> Scene:
    """One isotropic Gaussian whose mean projects exactly onto the centre of
    pixel (px,py); no mesh."""
    cam = _identity_cam(w, h, f)
    x = (px + 0.5 - cam.cx) / f * z
    y = (py + 0.5 - cam.cy) / f * z
    g = Gaussians(np.array([[x, y, z]], np.float32), np.full((1, 3), scale, np.float32),
                  np.array([[1, 0, 0, 0]], np.float32), np.array([opacity], np.float32),
                  np.array([[sh_dc]], np.float32), 0)
    return Scene("micro_lone", 0, g, None, [cam])


def micro_two_gaussians(z1=2.0, z2=2.5, o1=0.5, o2=0.7, w=32, h=32, f=32.0) -> Scene:
    """Two Gaussians centred on the same pixel at depths z1 and z2."""
    cam = _identity_cam(w, h, f)
    px, py = 16, 16
    ms = []
    for z in (z1, z2):
        ms.append([(px + 0.5 - cam.cx) / f * z, (py + 0.5 - cam.cy) / f * z, z])
    g = Gaussians(np.array(ms, np.float32), np.full((2, 3), 0.05, np.float32),
                  np.array([[1, 0, 0, 0]] * 2, np.float32), np.array([o1, o2], np.float32),
                  np.array([[[0.2, 0.4, 0.6]], [[0.9, 0.1, 0.3]]], np.float32), 0)
    return Scene("micro_two", 0, g, None, [cam])


def micro_quad_only(tex=None, w=32, h=32, f=32.0, z=3.0, seed=5) -> Scene:
    """A quad filling the view at depth z, no Gaussians."""
    cam = _identity_cam(w, h, f)
    s = 1.2 * (w / 2.0) / f * z
    verts = np.array([[-s, -s, z], [s, -s, z], [s, s, z], [-s, s, z]], np.float32)
    uvs = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    faces = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    if tex is None:
        tex = np.random.default_rng(seed).integers(0, 256, (16, 16, 3), dtype=np.uint8)
    empty = Gaussians(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
                      np.zeros((0, 4), np.float32), np.zeros(0, np.float32),
                      np.zeros((0, 1, 3), np.float32), 0)
    return Scene("micro_quad", 0, empty, Mesh(verts, uvs, faces, tex), [cam])


def with_fields(obj, **kw):
    return dataclasses.replace(obj, **kw)


# --------------------------------------------------------------------------
# prior normal maps for the mesh-pruning metrics (stand-ins for the monocular
# normal prior the paper takes from a pre-trained model)
# --------------------------------------------------------------------------

def prior_normal_maps(cameras, seed: int = 0, cutoff_px: float = 4.0, strength: float = 0.6,
                      n_patches: int = 6):
    """Per camera a planar [3, H, W] float32 field of unit normals: a smooth
    field (band-limited noise of ``cutoff_px`` correlation length around the
    view axis, tilted by ``strength``) with ``n_patches`` rectangles of
    high-frequency noise (where a prior would see clutter)."""
    rng = np.random.default_rng(seed)
    out = []
    for cam in cameras:
        W, H = int(cam.width), int(cam.height)
        size = 1 << int(np.ceil(np.log2(max(W, H))))
        field = _band_limited_noise(rng, size, cutoff_px)[:H, :W].astype(np.float64) / 255.0 - 0.5
        n = np.empty((3, H, W))
        n[0] = strength * field[..., 0]
        n[1] = strength * field[..., 1]
        n[2] = -1.0 + 0.2 * field[..., 2]
        for _ in range(n_patches):
            w, h = int(rng.integers(4, max(5, W // 6))), int(rng.integers(4, max(5, H // 6)))
            x, y = int(rng.integers(0, max(1, W - w))), int(rng.integers(0, max(1, H - h)))
            n[:, y:y + h, x:x + w] += rng.normal(0.0, 0.5, (3, h, w))
        n /= np.linalg.norm(n, axis=0, keepdims=True)
        out.append(n.astype(np.float32))
    return out
