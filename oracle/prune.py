"""Oracle of the mesh-pruning metrics (TEST INFRASTRUCTURE ONLY).

Sec. 3.3 and Algorithm 1 (stage 1) prune the extracted mesh before the joint
optimisation with three per-triangle metrics, combined as M_P = M_N && M_A &&
M_S, then drop small connected pieces:
  * normal variation (M_N): per training view, the alpha_normal percent of
    pixels with the highest total variation of a prior normal map mark the
    triangle they see (pixel -> triangle from the mesh raster) for removal;
  * adjacent angle (M_A): a triangle whose normal differs by more than 45
    degrees from an adjacent triangle's is removed;
  * area (M_S): the alpha_area percent smallest triangles are removed;
  * group: kept triangles in edge-connected pieces of fewer than alpha_group
    triangles are removed.
Defaults (supplementary implementation details): alpha_normal 20, alpha_area
50, alpha_group 100.

Readings (the paper leaves them open), shared with the GPU path:
  * M_N, M_A, M_S are keep masks, so && keeps a triangle only if no metric
    removes it (the text's "marked for removal" by any metric);
  * the prior normal map is an input ([3][H][W] per view, planar; the
    StableNormal model is not available), its total variation at pixel
    (x, y) is sum_c (|N_c(x+1,y) - N_c(x,y)| + |N_c(x,y+1) - N_c(x,y)|) with
    absent neighbours contributing 0, evaluated in FP32 in that order (it
    decides an integer ranking, so both sides take it in the kernel's
    precision); per view the k = floor(alpha_normal * C / 100) covered pixels
    (tri_id >= 0, C of them) ranking first by (TV descending, pixel index
    ascending) mark their triangles;
  * a triangle's normal is (v1 - v0) x (v2 - v0) in FP64 (winding as given),
    adjacency is a shared edge (unordered vertex pair), and the angle test is
    n_f . n_g < cos(45 deg) |n_f| |n_g|, evaluated as
    dot < cos45 * sqrt(|n_f|^2 * |n_g|^2) in FP64; zero-area triangles take
    no part in it;
  * area ranks by (|n_f|^2, index) with |n_f|^2 computed in FP64 as
    ((cx * cx) + (cy * cy)) + (cz * cz), cx = ay bz - az by etc. without
    fused operations (bit-identical on both sides); the first
    floor(alpha_area * F / 100) are removed;
  * groups: components of the kept triangles under shared edges between kept
    triangles, labelled by their smallest triangle index; pieces with fewer
    than alpha_group triangles are removed.
Hole closing and LS3 smoothing (the later steps of stage 1) are out of scope.

Outputs: flags per triangle (bit 1 normal, 2 angle, 4 area, 8 group),
keep = flags == 0, and the component label (-1 where a metric removed it).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

F_NORMAL, F_ANGLE, F_AREA, F_GROUP = 1, 2, 4, 8


def face_normals(verts, faces):
    """FP64 (v1 - v0) x (v2 - v0) per face and its squared norm, in the
    operation order of the readings."""
    v = np.asarray(verts, np.float32).astype(np.float64)
    f = np.asarray(faces, np.int64)
    a = v[f[:, 1]] - v[f[:, 0]]
    b = v[f[:, 2]] - v[f[:, 0]]
    cx = a[:, 1] * b[:, 2] - a[:, 2] * b[:, 1]
    cy = a[:, 2] * b[:, 0] - a[:, 0] * b[:, 2]
    cz = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    n2 = (cx * cx + cy * cy) + cz * cz
    return np.stack([cx, cy, cz], 1), n2


def edge_pairs(faces):
    """All (f, g) pairs, f < g, of triangles sharing an edge (an unordered
    vertex pair; every pair of the triangles on a non-manifold edge)."""
    f = np.asarray(faces, np.int64)
    F = len(f)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    e.sort(1)
    owner = np.tile(np.arange(F), 3)
    order = np.lexsort((owner, e[:, 1], e[:, 0]))
    e, owner = e[order], owner[order]
    if len(e) == 0:
        return np.zeros((0, 2), np.int64)
    new_grp = np.concatenate([[True], (e[1:, 0] != e[:-1, 0]) | (e[1:, 1] != e[:-1, 1])])
    starts = np.nonzero(new_grp)[0]
    ends = np.concatenate([starts[1:], [len(e)]])
    pairs = []
    two = (ends - starts) == 2
    a, b = owner[starts[two]], owner[starts[two] + 1]
    keep = a != b
    pairs.append(np.stack([np.minimum(a, b)[keep], np.maximum(a, b)[keep]], 1))
    for s0, e0 in zip(starts[~two], ends[~two]):
        grp = np.unique(owner[s0:e0])
        for x in range(len(grp)):
            for y in range(x + 1, len(grp)):
                pairs.append(np.array([[grp[x], grp[y]]]))
    out = np.concatenate(pairs) if pairs else np.zeros((0, 2), np.int64)
    return np.unique(out, axis=0) if len(out) else out.reshape(0, 2)


def normal_tv(nmap):
    """FP32 total variation of a [3, H, W] normal map (readings' order)."""
    N = np.asarray(nmap, np.float32)
    _, H, W = N.shape
    tv = np.zeros((H, W), np.float32)
    for c in range(3):
        dx = np.zeros((H, W), np.float32)
        dy = np.zeros((H, W), np.float32)
        dx[:, :-1] = np.abs(N[c, :, 1:] - N[c, :, :-1])
        dy[:-1, :] = np.abs(N[c, 1:, :] - N[c, :-1, :])
        tv = tv + (dx + dy)
    return tv


def prune(verts, faces, tri_ids, normal_maps, alpha_normal=20.0, alpha_area=50.0, angle_deg=45.0,
          alpha_group=100):
    """tri_ids: per view [H*W] int (-1: no triangle); normal_maps: per view
    [3, H, W].  Returns (flags uint8 [F], keep bool [F], label int64 [F])."""
    F = len(faces)
    flags = np.zeros(F, np.uint8)
    # normal-variation marks
    for tri, nm in zip(tri_ids, normal_maps):
        tri = np.asarray(tri, np.int64).reshape(-1)
        tv = normal_tv(nm).reshape(-1)
        cov = np.nonzero(tri >= 0)[0]
        k = int(np.floor(alpha_normal * len(cov) / 100.0))
        if k > 0:
            order = np.lexsort((cov, -tv[cov].astype(np.float64)))   # TV descending, index ascending
            flags[tri[cov[order[:k]]]] |= F_NORMAL
    # adjacent angles
    nrm, n2 = face_normals(verts, faces)
    pairs = edge_pairs(faces)
    cos_t = math.cos(float(angle_deg) * (math.pi / 180.0))
    if len(pairs):
        f, g = pairs[:, 0], pairs[:, 1]
        ok = (n2[f] > 0) & (n2[g] > 0)
        dot = (nrm[f, 0] * nrm[g, 0] + nrm[f, 1] * nrm[g, 1]) + nrm[f, 2] * nrm[g, 2]
        sharp = ok & (dot < cos_t * np.sqrt(n2[f] * n2[g]))
        flags[f[sharp]] |= F_ANGLE
        flags[g[sharp]] |= F_ANGLE
    # smallest areas
    k = int(np.floor(alpha_area * F / 100.0))
    if k > 0:
        order = np.lexsort((np.arange(F), n2))
        flags[order[:k]] |= F_AREA
    # small connected pieces of what is kept
    keep0 = flags == 0
    label = np.full(F, -1, np.int64)
    idx = np.nonzero(keep0)[0]
    if len(idx):
        if len(pairs):
            both = keep0[pairs[:, 0]] & keep0[pairs[:, 1]]
            p = pairs[both]
        else:
            p = np.zeros((0, 2), np.int64)
        A = coo_matrix((np.ones(len(p)), (p[:, 0], p[:, 1])), shape=(F, F))
        _, comp = connected_components(A, directed=False)
        comp_k = comp[idx]
        # label = smallest triangle index in the component
        first = {}
        for fi, c in zip(idx, comp_k):
            if c not in first:
                first[c] = fi
        label[idx] = [first[c] for c in comp_k]
        sizes = np.bincount(comp_k, minlength=comp.max() + 1)
        small = sizes[comp_k] < alpha_group
        flags[idx[small]] |= F_GROUP
    keep = flags == 0
    return flags, keep, label
