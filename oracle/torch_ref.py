"""FP64 PyTorch-CPU restatement of the hybrid renderer, used as the gradient
oracle (TEST INFRASTRUCTURE ONLY).

The forward mirrors ``hm_oracle.c`` step by step (Eq. 1, Sec. 3.1 covariance
and EWA projection, Eq. 2 blending, the Sec. 3.4 mesh cut-off and composite)
with plain tensor ops in float64; gradients are the exact derivative of that
forward, obtained with autograd.  Discrete decisions (which Gaussians are
blended at a pixel, the stop point, the mesh hit and its UV) carry no
gradient, exactly as in the renderer's backward: Sec. 3.4 makes the texture
map optimisable while vertex positions are not optimised (Sec. 5).

Decisions are taken on detached FP64 values; the sort order and the mesh pass
(tri_id, depth, uv) come from the C oracle.
"""
from __future__ import annotations

import math
from types import SimpleNamespace

import numpy as np
import torch

from . import oracle as O

DT = torch.float64


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=DT)


# --------------------------------------------------------------------------
# real SH basis in Cartesian form: for m > 0
#   Y_l^m  = sqrt(2) K_l^m (-1)^m Re((x+iy)^m) d^m/dz^m P_l(z)
#   Y_l^-m = sqrt(2) K_l^m (-1)^m Im((x+iy)^m) d^m/dz^m P_l(z)
#   Y_l^0  = K_l^0 P_l(z)
# which equals the associated-Legendre form (Condon-Shortley phase) because
# sin^m(theta) cos(m phi) = Re((x+iy)^m) on the unit sphere.
# --------------------------------------------------------------------------

def _legendre_deriv_coeffs(l, m):
    c = np.zeros(l + 1)
    c[l] = 1.0
    p = np.polynomial.legendre.leg2poly(c)          # power-series coefficients of P_l
    p = np.polynomial.polynomial.polyder(p, m) if m > 0 else p
    return p


def sh_basis_torch(deg, d):
    """d: [N,3] unit directions -> [N,(deg+1)^2]."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    cols = [None] * ((deg + 1) ** 2)
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, deg + 1):
        re.append(re[-1] * x - im[-1] * y)
        im.append(re[-2] * y + im[-1] * x)
    for l in range(deg + 1):
        for m in range(0, l + 1):
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            coef = _legendre_deriv_coeffs(l, m)
            poly = torch.zeros_like(z)
            for k in range(len(coef) - 1, -1, -1):
                poly = poly * z + float(coef[k])
            if m == 0:
                cols[l * l + l] = K * poly
            else:
                s = math.sqrt(2.0) * K * (-1.0) ** m
                cols[l * l + l + m] = s * re[m] * poly
                cols[l * l + l - m] = s * im[m] * poly
    return torch.stack(cols, 1)


# --------------------------------------------------------------------------
# projection
# --------------------------------------------------------------------------

def quat_to_rot(q):
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1),
    ], 1)


def project_torch(cam, means, scales, quats, sh, sh_degree, filt3d=None, kernel2d=0.3, antialias=False):
    """Differentiable projection of every Gaussian (visibility decided
    elsewhere).  Returns mean2d [N,2], conic [N,3] (xx,xy,yy), color [N,3]
    and the opacity factor [N] of the Mip-Splatting filters (1 without them;
    the 3D filter variance ``filt3d`` is a constant, not differentiated)."""
    c = O.cam_array(cam)
    Rc = _t(c[:9].reshape(3, 3))
    tc = _t(c[9:12])
    fx, fy, cx, cy = (float(v) for v in c[12:16])
    W, H = int(cam.width), int(cam.height)
    p = means @ Rc.T + tc
    tx, ty, tz = p.unbind(1)
    limx, limy = 1.3 * (0.5 * W / fx), 1.3 * (0.5 * H / fy)
    txz = torch.clamp(tx / tz, -limx, limx)
    tyz = torch.clamp(ty / tz, -limy, limy)
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, zero, -fx * txz / tz], 1),
                     torch.stack([zero, fy / tz, -fy * tyz / tz], 1)], 1)        # [N,2,3]
    Rq = quat_to_rot(quats)
    if filt3d is not None:
        v = _t(filt3d)[:, None]
        s_eff = torch.sqrt(scales * scales + v)                 # Sigma + v I = R diag(s^2 + v) R^T
        rho3 = torch.prod(scales / s_eff, dim=1)
    else:
        s_eff = scales
        rho3 = torch.ones_like(tz)
    M = Rq * s_eff[:, None, :]
    Sig = M @ M.transpose(1, 2)
    T = J @ Rc                                                                      # [N,2,3]
    S2 = T @ Sig @ T.transpose(1, 2)
    a = S2[:, 0, 0] + kernel2d
    b = S2[:, 0, 1]
    cc = S2[:, 1, 1] + kernel2d
    det = a * cc - b * b
    conic = torch.stack([cc / det, -b / det, a / det], 1)
    if antialias:
        det0 = S2[:, 0, 0] * S2[:, 1, 1] - b * b
        rho2 = torch.sqrt(torch.clamp(det0, min=0.0) / det)
    else:
        rho2 = torch.ones_like(tz)
    mean2d = torch.stack([fx * tx / tz + cx, fy * ty / tz + cy], 1)
    C = -(Rc.T @ tc)
    d = means - C
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    Y = sh_basis_torch(sh_degree, d)                                                # [N,K]
    col = 0.5 + torch.einsum("nk,nkc->nc", Y, sh)
    col = torch.clamp(col, min=0.0)
    return mean2d, conic, col, rho3 * rho2


# --------------------------------------------------------------------------
# texture
# --------------------------------------------------------------------------

def bilinear_torch(tex, u, v):
    """tex [th,tw,3] tensor; u,v [P] (no gradient) -> [P,3]; clamp-to-edge."""
    th, tw = tex.shape[:2]
    s = u * tw - 0.5
    t = v * th - 0.5
    x0 = torch.floor(s)
    y0 = torch.floor(t)
    fx = (s - x0)[:, None]
    fy = (t - y0)[:, None]
    x0 = x0.long()
    y0 = y0.long()

    def tx(xi, yi):
        return tex[yi.clamp(0, th - 1), xi.clamp(0, tw - 1)]
    return ((1 - fx) * (1 - fy) * tx(x0, y0) + fx * (1 - fy) * tx(x0 + 1, y0)
            + (1 - fx) * fy * tx(x0, y0 + 1) + fx * fy * tx(x0 + 1, y0 + 1))


# --------------------------------------------------------------------------
# blend for a set of pixels
# --------------------------------------------------------------------------

def blend_torch(pxy, mean2d, conic, opacity, color, depth_f32, order, hit, Dm, Im):
    """pxy [P,2] pixel centres; per-Gaussian tensors over all N; ``order``:
    visible Gaussians sorted by (depth, index); hit [P] bool, Dm [P] float32
    numpy, Im [P,3] tensor.  Returns rgb [P,3], T [P]."""
    idx = torch.as_tensor(order, dtype=torch.long)
    mx = mean2d[idx, 0]
    my = mean2d[idx, 1]
    ca, cb, cc = conic[idx, 0], conic[idx, 1], conic[idx, 2]
    o = opacity[idx]
    col = color[idx]
    dz = torch.as_tensor(np.asarray(depth_f32)[order].astype(np.float32))
    dx = pxy[:, 0:1] - mx[None, :]
    dy = pxy[:, 1:2] - my[None, :]
    d2 = ca[None] * dx * dx + 2.0 * cb[None] * dx * dy + cc[None] * dy * dy
    araw = o[None] * torch.exp(-0.5 * d2)
    with torch.no_grad():
        behind = torch.as_tensor(hit)[:, None] & (dz[None, :] >= torch.as_tensor(Dm)[:, None])
        elig = (~behind) & (d2 <= 9.0) & (araw >= 1.0 / 255.0)
    a = torch.where(elig, torch.clamp(araw, max=0.99), torch.zeros_like(araw))
    with torch.no_grad():
        Tincl = torch.cumprod(1.0 - a, 1)
        stop = Tincl < 1e-4
        keep = torch.cumsum(stop.to(torch.int64), 1) == 0
    a = a * keep
    Tin = torch.cumprod(1.0 - a, 1)
    Tex = torch.cat([torch.ones_like(Tin[:, :1]), Tin[:, :-1]], 1)
    w = a * Tex
    rgb = w @ col + Tin[:, -1:] * Im if Tin.shape[1] else Im.clone()
    T = Tin[:, -1] if Tin.shape[1] else torch.ones(pxy.shape[0], dtype=DT)
    return rgb, T


def render_grad(scene, view, gI, gT=None, pix=None, gaussians=None, tex=None, chunk=1024, filt3d=None,
                kernel2d=0.3, antialias=False):
    """Gradient of L = sum_p gI[:,p] . I_h(p) + gT[p] T(p) over the listed
    pixels (all if None) of one view, with respect to means, scales, quats,
    opacity, sh (all as given, i.e. activated) and, if the scene has a mesh,
    the texels.  Returns (loss, grads dict)."""
    cam = scene.cameras[view]
    g = scene.gaussians if gaussians is None else gaussians
    W, H = int(cam.width), int(cam.height)
    if pix is None:
        pix = np.arange(W * H, dtype=np.int64)
    pix = np.asarray(pix, np.int64)
    bg = np.asarray(scene.bg, np.float64)
    texture = None
    if scene.mesh is not None:
        texture = O.texture_unit(scene.mesh.texture) if tex is None else np.asarray(tex, np.float64)
        mr = O.mesh_raster(cam, scene.mesh, bg=bg, pix=pix, tex=texture)
    else:
        mr = O.empty_mesh_result(len(pix), bg)
    pr = O.project(cam, g, filt3d=filt3d, kernel2d=kernel2d, antialias=antialias)
    order = O.sort_order(pr)

    means = _t(g.means).requires_grad_()
    scales = _t(g.scales).requires_grad_()
    quats = _t(g.quats).requires_grad_()
    opac = _t(g.opacity).requires_grad_()
    sh = _t(np.asarray(g.sh).astype(np.float64)).requires_grad_()
    texT = _t(texture).requires_grad_() if texture is not None else None
    mean2d, conic, color, osc = project_torch(cam, means, scales, quats, sh, g.sh_degree, filt3d=filt3d,
                                              kernel2d=kernel2d, antialias=antialias)
    opac_eff = opac * osc
    # blend against detached leaves, then push their gradients through the projection
    l_m2 = mean2d.detach().requires_grad_()
    l_co = conic.detach().requires_grad_()
    l_cl = color.detach().requires_grad_()
    l_op = opac_eff.detach().requires_grad_()
    gI = np.asarray(gI, np.float64).reshape(3, -1)
    gT = np.zeros(len(pix)) if gT is None else np.asarray(gT, np.float64)
    loss = 0.0
    hit_all = mr.tri_id >= 0
    for s in range(0, len(pix), chunk):
        e = min(len(pix), s + chunk)
        q = pix[s:e]
        pxy = _t(np.stack([q % W + 0.5, q // W + 0.5], 1))
        hit = hit_all[s:e]
        Im = _t(np.repeat(bg[None], e - s, 0))
        if texT is not None and hit.any():
            hi = np.nonzero(hit)[0]
            Imh = bilinear_torch(texT, _t(mr.uv[0, s:e][hi]), _t(mr.uv[1, s:e][hi]))
            Im = Im.index_put((torch.as_tensor(hi),), Imh)
        rgb, T = blend_torch(pxy, l_m2, l_co, l_op, l_cl, pr.depth, order, hit,
                             mr.depth[s:e], Im)
        L = (rgb * _t(gI[:, s:e].T)).sum() + (T * _t(gT[s:e])).sum()
        L.backward()
        loss += float(L.detach())
    outs, grads = [mean2d, conic, color, opac_eff], [l_m2.grad, l_co.grad, l_cl.grad, l_op.grad]
    keep = [(o, gr) for o, gr in zip(outs, grads) if gr is not None]
    torch.autograd.backward([o for o, _ in keep], [gr for _, gr in keep])
    leaves = dict(means=(means, g.means), scales=(scales, g.scales), quats=(quats, g.quats),
                  opacity=(opac, g.opacity), sh=(sh, g.sh))
    if texT is not None:
        leaves["texture"] = (texT, texture)
    res = {k: (np.zeros(np.shape(ref)) if t.grad is None else t.grad.numpy())
           for k, (t, ref) in leaves.items()}
    return loss, res


def render_forward(scene, view, pix=None, gaussians=None, tex=None, filt3d=None, kernel2d=0.3,
                   antialias=False):
    """Forward only (for cross-checking against the C oracle)."""
    cam = scene.cameras[view]
    g = scene.gaussians if gaussians is None else gaussians
    W, H = int(cam.width), int(cam.height)
    if pix is None:
        pix = np.arange(W * H, dtype=np.int64)
    bg = np.asarray(scene.bg, np.float64)
    if scene.mesh is not None:
        texture = O.texture_unit(scene.mesh.texture) if tex is None else np.asarray(tex, np.float64)
        mr = O.mesh_raster(cam, scene.mesh, bg=bg, pix=pix, tex=texture)
    else:
        texture = None
        mr = O.empty_mesh_result(len(pix), bg)
    pr = O.project(cam, g, filt3d=filt3d, kernel2d=kernel2d, antialias=antialias)
    order = O.sort_order(pr)
    with torch.no_grad():
        mean2d, conic, color, osc = project_torch(cam, _t(g.means), _t(g.scales), _t(g.quats),
                                                  _t(np.asarray(g.sh).astype(np.float64)), g.sh_degree,
                                                  filt3d=filt3d, kernel2d=kernel2d, antialias=antialias)
        q = np.asarray(pix)
        pxy = _t(np.stack([q % W + 0.5, q // W + 0.5], 1))
        hit = mr.tri_id >= 0
        Im = _t(mr.rgb.T.copy())
        rgb, T = blend_torch(pxy, mean2d, conic, _t(g.opacity) * osc, color, pr.depth, order, hit,
                             mr.depth, Im)
    return SimpleNamespace(rgb=rgb.numpy().T, T=T.numpy(), mesh=mr, proj=pr)
