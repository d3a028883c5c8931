"""Pins of the mesh-pruning oracle (Sec. 3.3, Algorithm 1 stage 1): closed
forms on small meshes whose answers follow from their geometry -- flat grids
(no sharp edges, equal areas), a cube (every triangle borders a 90 degree
edge), hinged strips at 30 and 60 degrees, triangles of known areas, disjoint
pieces of known sizes -- and normal maps with known total variation."""
import numpy as np

from oracle import prune as P


def grid(nx, ny, z=0.0, x0=0.0, flip=False):
    """Flat (nx x ny)-quad grid in the plane z, two triangles per quad,
    counter-clockwise seen from +z (normals +z) unless flip."""
    xs, ys = np.meshgrid(np.arange(nx + 1, dtype=np.float32), np.arange(ny + 1, dtype=np.float32))
    v = np.stack([xs.ravel() + x0, ys.ravel(), np.full(xs.size, z, np.float32)], 1)
    f = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, d = a + 1, a + nx + 1, a + nx + 2
            t1, t2 = (a, b, d), (a, d, c)
            if flip:
                t1, t2 = t1[::-1], t2[::-1]
            f += [t1, t2]
    return v, np.array(f, np.int64)


def test_flat_grid_has_no_sharp_edges_and_equal_areas():
    v, f = grid(6, 5)
    nrm, n2 = P.face_normals(v, f)
    assert np.all(n2 == 1.0) and np.all(nrm[:, 2] == 1.0)
    flags, keep, label = P.prune(v, f, [], [], alpha_area=50.0, alpha_group=1)
    assert not np.any(flags & P.F_ANGLE)
    # equal areas: the first floor(0.5 F) by index are the smallest
    assert np.array_equal(np.nonzero(flags & P.F_AREA)[0], np.arange(len(f) // 2))


def test_cube_every_triangle_borders_a_right_angle():
    v = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], np.float32)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    f = np.array([t for a, b, c, d in quads for t in ((a, b, c), (a, c, d))], np.int64)
    nrm, n2 = P.face_normals(v, f)
    # outward normals: the face centroid minus the cube centre points along them
    cen = v[f].mean(1) - 0.5
    assert np.all((nrm * cen).sum(1) > 0)
    flags, keep, _ = P.prune(v, f, [], [], alpha_area=0.0, alpha_group=1)
    assert np.all(flags & P.F_ANGLE) and not keep.any()
    assert len(P.edge_pairs(f)) == 18          # 12 triangles x 3 edges / 2


def _hinge(deg):
    """Two 3x1-quad strips sharing the edge x = 0, the second tilted by deg."""
    t = np.deg2rad(deg)
    v, f = grid(3, 1)
    v2 = v.copy()
    v2[:, 0] = -v[:, 0] * np.cos(t)
    v2[:, 2] = v[:, 0] * np.sin(t)
    n = len(v)
    f2 = f[:, ::-1] + n                       # mirrored in x: flip to keep the winding consistent
    verts = np.concatenate([v, v2]).astype(np.float32)
    # weld the shared edge (x = 0) of the two strips
    remap = np.arange(2 * n)
    for i in range(n):
        if v[i, 0] == 0:
            remap[n + i] = i
    return verts, remap[np.concatenate([f, f2])]


def test_hinge_angle_threshold():
    for deg, sharp in ((30.0, False), (60.0, True)):
        v, f = _hinge(deg)
        flags, _, _ = P.prune(v, f, [], [], alpha_area=0.0, alpha_group=1)
        hit = np.nonzero(flags & P.F_ANGLE)[0]
        if sharp:
            # exactly the two triangles touching the hinge edge on each side
            assert len(hit) == 2
            touch = [i for i in range(len(f)) if sum(v[f[i], 0] == 0) == 2]
            assert sorted(hit) == sorted(touch)
        else:
            assert len(hit) == 0


def test_area_ranking_of_known_triangles():
    # right triangles with legs (a, b): |n|^2 = (a b)^2
    legs = [(2, 3), (1, 1), (4, 1), (1, 1), (3, 3), (0.5, 2)]
    v, f = [], []
    for k, (a, b) in enumerate(legs):
        base = len(v)
        v += [(10 * k, 0, 0), (10 * k + a, 0, 0), (10 * k, b, 0)]
        f.append((base, base + 1, base + 2))
    v = np.array(v, np.float32)
    f = np.array(f, np.int64)
    _, n2 = P.face_normals(v, f)
    assert np.allclose(n2, [(a * b) ** 2 for a, b in legs])
    flags, _, _ = P.prune(v, f, [], [], alpha_area=50.0, alpha_group=1)
    # 3 smallest by (area, index): the two unit triangles (1, 3) then 0.5 x 2 (5)
    assert sorted(np.nonzero(flags & P.F_AREA)[0]) == [1, 3, 5]


def test_small_pieces_are_removed():
    v1, f1 = grid(5, 5)                       # 50 triangles
    v2, f2 = grid(15, 5, x0=100.0)            # 150 triangles
    v = np.concatenate([v1, v2])
    f = np.concatenate([f1, f2 + len(v1)])
    flags, keep, label = P.prune(v, f, [], [], alpha_area=0.0, alpha_group=100)
    assert np.all(flags[:50] == P.F_GROUP) and np.all(keep[50:])
    assert np.all(label[:50] == 0) and np.all(label[50:] == 50)


def test_normal_tv_closed_forms_and_marks():
    H, W = 6, 8
    const = np.zeros((3, H, W), np.float32)
    const[2] = 1.0
    assert np.all(P.normal_tv(const) == 0.0)
    step = const.copy()
    step[0, :, 5:] = 0.6
    step[2, :, 5:] = 0.8                       # a crease between columns 4 and 5
    tv = P.normal_tv(step)
    assert np.all(tv[:, 4] == np.float32(0.6) + np.float32(0.2))
    assert np.count_nonzero(tv) == H
    # covered pixels see triangle (x // 2); 20% of 48 covered = 9 marks: the
    # 6 crease pixels (column 4 -> triangle 2) and then, at TV 0, the 3 lowest
    # pixel indices (row 0, columns 0..2 -> triangles 0, 0, 1)
    tri = np.tile(np.arange(W) // 2, H)
    v, f = grid(2, 2)                         # 8 triangles, only the ids matter
    flags, _, _ = P.prune(v, f, [tri], [step], alpha_normal=20.0, alpha_area=0.0, alpha_group=1)
    assert sorted(np.nonzero(flags & P.F_NORMAL)[0]) == [0, 1, 2]
