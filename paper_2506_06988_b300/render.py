"""Hybrid mesh-Gaussian rendering on one GPU through the libhm C ABI.

``Renderer`` owns the device buffers for a fixed set of cameras and scene
sizes and runs the four stages of a frame on the current CUDA stream:

    hm_rasterize_mesh     I_m, D_m, per-tile farthest mesh depth
    hm_project_gaussians  per (camera, Gaussian) records
    hm_bin_sort           (tile, depth)-sorted pairs and tile ranges
    hm_blend_forward      I_h = I_gs + T * back (Eq. 2 with the Sec. 3.4 cut-off)

and ``hm_blend_backward`` for gradients.  PyTorch provides memory and the
stream; every step of the path runs in libhm's kernels.  ``HybridRender`` is
the ``torch.autograd.Function`` over it (activations such as exp/sigmoid of
the raw parameters stay in PyTorch).

Pair and work-item capacities grow on demand: a frame whose device status
reports HM_DEV_CAPACITY is re-run with the reported need (``render``); the
asynchronous ``forward`` leaves the check to the caller (``status``).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import lib

__all__ = ["MeshInput", "Renderer", "ChunkedRenderer", "HybridRender", "GraphStep"]


@dataclass
class MeshInput:
    verts: torch.Tensor      # [V,3] f32
    uvs: torch.Tensor        # [V,2] f32
    faces: torch.Tensor      # [F,3] i32
    texture: torch.Tensor    # [H,W,3] u8 or f32

    @property
    def tex_format(self) -> int:
        return lib.HM_TEX_RGBF32 if self.texture.dtype == torch.float32 else lib.HM_TEX_RGB8

    @staticmethod
    def from_numpy(m, device="cuda") -> "MeshInput":
        return MeshInput(torch.as_tensor(m.verts, dtype=torch.float32, device=device).contiguous(),
                         torch.as_tensor(m.uvs, dtype=torch.float32, device=device).contiguous(),
                         torch.as_tensor(m.faces, dtype=torch.int32, device=device).contiguous(),
                         torch.as_tensor(m.texture, device=device).contiguous())


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Renderer:
    """Buffers and stage launches for a fixed camera set and scene size.

    Per-pixel outputs (``rgb`` planar per camera, ``T``, ``n_contrib``,
    ``last_idx``, mesh ``tri_id``/``depth``/``mesh_rgb``/``uv``) are flat
    tensors over the concatenated pixels of all cameras; ``image(k)`` gives
    camera k's [3,H,W] view of ``rgb``.
    """

    def __init__(self, cams, n: int, sh_degree: int, *, sh_f16: bool = False,
                 n_verts: int = 0, n_faces: int = 0, tex_shape=None, tile=(16, 16),
                 batch: Optional[int] = None, mesh_cull: bool = True, bg=(0.0, 0.0, 0.0),
                 pair_capacity: Optional[int] = None, item_capacity: Optional[int] = None,
                 ellipse_cull: bool = True, pixel_buffers: Optional[dict] = None, mip: bool = False,
                 persistent: bool = False, device="cuda"):
        lib.load()
        self.device = torch.device(device)
        self.cam_list = list(cams)
        self.cams = lib.cameras(self.cam_list)
        self.V = len(self.cam_list)
        self.n = int(n)
        self.sh_degree = int(sh_degree)
        self.K = (self.sh_degree + 1) ** 2
        self.sh_format = lib.HM_SH_F16 if sh_f16 else lib.HM_SH_F32
        self.opt = lib.options(tile=tile, batch=batch, mesh_cull=mesh_cull, bg=bg,
                               ellipse_cull=ellipse_cull, mip=mip, persistent=persistent)
        # Mip-Splatting back-end (mip=True): the 2D Mip filter in the options and
        # the per-Gaussian 3D smoothing variance (set_filter_3d / mip_filter_3d)
        self.mip = bool(mip)
        self.filter_3d: Optional[torch.Tensor] = None
        self.bg = tuple(float(x) for x in bg)
        self.sizes = [(int(c.width), int(c.height)) for c in self.cam_list]
        self.pix_off = np.concatenate([[0], np.cumsum([w * h for w, h in self.sizes])]).astype(np.int64)
        self.npix = int(self.pix_off[-1])
        self.ntiles = lib.hm_total_tiles(self.cams, self.opt)
        if self.ntiles < 0:
            raise lib.HmError(lib.last_error())
        self.n_verts, self.n_faces = int(n_verts), int(n_faces)
        self.has_mesh = self.n_faces > 0 or tex_shape is not None
        self.tex_shape = tuple(tex_shape) if tex_shape is not None else None
        d = self.device
        f32, i32 = torch.float32, torch.int32
        M = self.V * self.n
        self.records = torch.empty(max(M, 1) * 12, dtype=f32, device=d)
        self.ranges = torch.empty(2 * self.ntiles, dtype=i32, device=d)
        self.n_pairs = torch.zeros(1, dtype=torch.int64, device=d)
        self.n_items = torch.zeros(1, dtype=torch.int64, device=d)
        self.status_word = torch.zeros(1, dtype=i32, device=d)
        self.work = torch.zeros(1, dtype=i32, device=d)      # tile counter of the persistent blend
        if pixel_buffers is not None:
            self.use_pixel_buffers(pixel_buffers)
        else:
            self.rgb = torch.empty(3 * self.npix, dtype=f32, device=d)
            self.T = torch.empty(self.npix, dtype=f32, device=d)
            self.n_contrib = torch.empty(self.npix, dtype=i32, device=d)
            self.last_idx = torch.empty(self.npix, dtype=i32, device=d)
            if self.has_mesh:
                self.tri_id = torch.empty(self.npix, dtype=i32, device=d)
                self.mesh_depth = torch.empty(self.npix, dtype=f32, device=d)
                self.mesh_rgb = torch.empty(3 * self.npix, dtype=f32, device=d)
                self.uv = torch.empty(2 * self.npix, dtype=f32, device=d)
                self.tile_max = torch.empty(self.ntiles, dtype=f32, device=d)
            else:
                self.tri_id = self.mesh_depth = self.mesh_rgb = self.uv = self.tile_max = None
        self._pair_cap = 0
        self._item_cap = 0
        self.set_pair_capacity(pair_capacity if pair_capacity else max(1024, 8 * M))
        if self.has_mesh:
            self.set_item_capacity(item_capacity if item_capacity else max(1024, 4 * self.V * self.n_faces))
        self.bwd_ws = None
        # side-stream overlap pays inside a CUDA graph (fork and join are
        # graph edges); launched eagerly the stream synchronisation costs more
        # than it hides, so it is off by default and on in GraphStep
        self.overlap = False
        self._side = None

    # per-pixel (and per-tile) storage: (name, elements per pixel or per tile, dtype)
    PIXEL_FIELDS = (("rgb", 3, torch.float32), ("T", 1, torch.float32), ("n_contrib", 1, torch.int32),
                    ("last_idx", 1, torch.int32))
    MESH_FIELDS = (("tri_id", 1, torch.int32), ("mesh_depth", 1, torch.float32),
                   ("mesh_rgb", 3, torch.float32), ("uv", 2, torch.float32))

    def use_pixel_buffers(self, bufs: dict):
        """Write the per-pixel outputs (and the per-tile farthest mesh depth)
        into caller tensors -- e.g. slices of larger arrays shared by several
        renderers -- instead of the renderer's own: keys as ``PIXEL_FIELDS``,
        ``MESH_FIELDS`` and ``tile_max``, flat, sized for these cameras."""
        fields = self.PIXEL_FIELDS + (self.MESH_FIELDS if self.has_mesh else ())
        for name, per, dt in fields:
            t = bufs[name]
            if t.dtype != dt or t.numel() != per * self.npix or not t.is_contiguous():
                raise ValueError(f"pixel buffer {name}: need {per * self.npix} contiguous {dt}")
            setattr(self, name, t)
        if self.has_mesh:
            t = bufs["tile_max"]
            if t.dtype != torch.float32 or t.numel() != self.ntiles:
                raise ValueError(f"tile_max: need {self.ntiles} float32")
            self.tile_max = t
        else:
            self.tri_id = self.mesh_depth = self.mesh_rgb = self.uv = self.tile_max = None

    def retarget(self, cams, bufs: dict):
        """Render another set of cameras of the same sizes (in order) with
        the same scratch (records, pair lists, workspaces)."""
        cams = list(cams)
        sizes = [(int(c.width), int(c.height)) for c in cams]
        if sizes != self.sizes:
            raise ValueError("retarget needs cameras of the same sizes")
        self.cam_list = cams
        self.cams = lib.cameras(cams)
        self.use_pixel_buffers(bufs)

    # -- capacities -------------------------------------------------------------
    def set_pair_capacity(self, cap: int):
        cap = int(min(max(cap, 1024), lib.HM_MAX_PAIRS))
        self._pair_cap = cap
        self.pair_vals = torch.empty(cap, dtype=torch.int32, device=self.device)
        nb = lib.hm_bin_sort_workspace_size(self.cams, self.n, cap, self.opt)
        self.bin_ws = torch.empty(nb, dtype=torch.uint8, device=self.device)

    def set_item_capacity(self, cap: int):
        cap = int(min(max(cap, 1024), lib.HM_MAX_PAIRS))
        self._item_cap = cap
        nb = lib.hm_rasterize_mesh_workspace_size(self.cams, self.n_verts, self.n_faces, cap, self.opt)
        self.raster_ws = torch.empty(nb, dtype=torch.uint8, device=self.device)

    @property
    def pair_capacity(self) -> int:
        return self._pair_cap

    # -- stages -----------------------------------------------------------------
    def rasterize_mesh(self, mesh: MeshInput):
        s = _stream()
        th, tw = mesh.texture.shape[:2]
        lib.check(lib.hm_rasterize_mesh(self.cams, mesh.verts, mesh.uvs, self.n_verts, mesh.faces,
                                        self.n_faces, mesh.texture, tw, th, mesh.tex_format,
                                        self.opt, self.tri_id, self.mesh_depth, self.mesh_rgb,
                                        self.uv, self.tile_max, self._item_cap, self.n_items,
                                        self.status_word, self.raster_ws, self.raster_ws.numel(), s),
                  "hm_rasterize_mesh")

    def mip_filter_3d(self, means, s2: float = 0.2, cams=None) -> torch.Tensor:
        """Compute (and keep for the projections) Mip-Splatting's 3D
        smoothing variance per Gaussian from ``cams`` (default: this
        renderer's cameras -- the training views)."""
        cams = self.cams if cams is None else lib.cameras(cams)
        if self.filter_3d is None or self.filter_3d.numel() != self.n:
            self.filter_3d = torch.empty(self.n, dtype=torch.float32, device=self.device)
        lib.check(lib.hm_mip_filter_3d(cams, self.n, means.contiguous(), float(s2), float(self.opt.near_gauss),
                                       self.filter_3d, _stream()), "hm_mip_filter_3d")
        return self.filter_3d

    def set_filter_3d(self, v: Optional[torch.Tensor]):
        """Use ``v`` ([n] float32, device) as the 3D smoothing variance (None: off)."""
        if v is not None and (v.dtype != torch.float32 or v.numel() != self.n or not v.is_contiguous()):
            raise ValueError(f"filter_3d: need {self.n} contiguous float32")
        self.filter_3d = v

    def project(self, means, scales, quats, opacity, sh):
        lib.check(lib.hm_project_gaussians(self.cams, self.n, means, scales, quats, opacity, sh,
                                           self.sh_degree, self.sh_format, self.opt, self.records,
                                           _stream(), filter_3d=self.filter_3d), "hm_project_gaussians")

    def bin_sort(self, mesh_cull: Optional[bool] = None):
        """Binning and the per-tile depth sort; ``mesh_cull`` False bins
        without the tiles' mesh depths (so it can run before the mesh pass
        ends): longer lists, the same images -- the blend cuts every pixel at
        its mesh depth and the culled pairs are a depth-sorted suffix."""
        cull = self.opt.mesh_cull if mesh_cull is None else int(bool(mesh_cull))
        tmax = self.tile_max if (self.has_mesh and cull) else None
        saved = self.opt.mesh_cull
        self.opt.mesh_cull = cull
        try:
            lib.check(lib.hm_bin_sort(self.cams, self.n, self.records, tmax, self.opt, self.pair_vals,
                                      self._pair_cap, self.n_pairs, self.ranges, self.status_word,
                                      self.bin_ws, self.bin_ws.numel(), _stream()), "hm_bin_sort")
        finally:
            self.opt.mesh_cull = saved

    def blend(self, eval_stats: Optional[torch.Tensor] = None):
        md = self.mesh_depth if self.has_mesh else None
        mr = self.mesh_rgb if self.has_mesh else None
        lib.check(lib.hm_blend_forward(self.cams, self.n, self.records, self.pair_vals, self.ranges,
                                       md, mr, self.opt, self.rgb, self.T, self.n_contrib,
                                       self.last_idx, eval_stats, self.status_word, _stream(),
                                       work=self.work),
                  "hm_blend_forward")

    def count_evaluations(self):
        """Re-run the blend of the last frame with the evaluation counters:
        (alpha evaluations, list entries examined) -- synchronises."""
        st = torch.zeros(2, dtype=torch.int64, device=self.device)
        self.blend(st)
        v = st.cpu().tolist()
        return int(v[0]), int(v[1])

    def _side_stream(self) -> torch.cuda.Stream:
        if self._side is None:
            self._side = torch.cuda.Stream(device=self.device)
        return self._side

    def _bin_stream(self) -> torch.cuda.Stream:
        """High-priority stream for the critical chains of an overlapped
        frame -- projection and binning (many short dependent kernels) in
        the forward, blend and projection gradients in the backward -- so
        their launches take SMs first while the mesh pass or the texel
        gradients on the current stream fill the rest."""
        if getattr(self, "_bin", None) is None:
            self._bin = torch.cuda.Stream(device=self.device, priority=-1)
        return self._bin

    def forward(self, means, scales, quats, opacity, sh, mesh: Optional[MeshInput] = None,
                overlap: Optional[bool] = None):
        """All four stages, asynchronously on the current stream.  With
        ``overlap`` (default ``self.overlap``) the projection and the binning
        (without the tile mesh cull, which would wait for the mesh pass) run
        on a high-priority side stream while the mesh pass runs on the
        current stream; the blend joins them -- inside a graph capture a
        fork and a join.  The images, counts and stop indices are the same
        either way."""
        self.status_word.zero_()
        if self.has_mesh and (self.overlap if overlap is None else overlap):
            main = torch.cuda.current_stream(self.device)
            hi = self._bin_stream()
            hi.wait_stream(main)
            with torch.cuda.stream(hi):
                self.project(means, scales, quats, opacity, sh)
                self.bin_sort(mesh_cull=False)
            self.rasterize_mesh(mesh)
            main.wait_stream(hi)
            self.blend()
            return
        else:
            if self.has_mesh:
                self.rasterize_mesh(mesh)
            self.project(means, scales, quats, opacity, sh)
        self.bin_sort()
        self.blend()

    def status(self):
        """(status bits, pair count, mesh work items) -- synchronises."""
        st, npairs, nitems = int(self.status_word.item()), int(self.n_pairs.item()), int(self.n_items.item())
        return st, npairs, nitems

    def render(self, means, scales, quats, opacity, sh, mesh: Optional[MeshInput] = None,
               max_retries: int = 3, overlap: Optional[bool] = None):
        """forward() plus the capacity check; grows the buffers and re-runs
        when a capacity was exceeded.  Raises on HM_DEV_TIMEOUT and
        HM_DEV_BAD_INDEX."""
        for _ in range(max_retries + 1):
            self.forward(means, scales, quats, opacity, sh, mesh, overlap=overlap)
            st, npairs, nitems = self.status()
            lib.check_device_status(st)
            if not st & lib.HM_DEV_CAPACITY:
                return self
            if npairs > self._pair_cap:
                self.set_pair_capacity(int(npairs * 1.25) + 1024)
            if self.has_mesh and nitems > self._item_cap:
                self.set_item_capacity(int(nitems * 1.25) + 1024)
        raise lib.HmError("capacity retries exhausted")

    def grad_buffers(self, tex_shape=None):
        d = self.device
        g = dict(means=torch.zeros(self.n, 3, device=d), scales=torch.zeros(self.n, 3, device=d),
                 quats=torch.zeros(self.n, 4, device=d), opacity=torch.zeros(self.n, device=d),
                 sh=torch.zeros(self.n, self.K, 3, device=d))
        if tex_shape is not None:
            g["texture"] = torch.zeros(tex_shape[0], tex_shape[1], 3, device=d)
        return g

    def backward(self, means, scales, quats, opacity, sh, dL_drgb, dL_dT=None,
                 mesh: Optional[MeshInput] = None, tex_grad: bool = False, out=None,
                 stages: int = 0, zero: bool = True, overlap: Optional[bool] = None,
                 dL_dmesh: Optional[torch.Tensor] = None):
        """Gradients of the last forward, accumulated into fresh zero tensors
        (or into ``out``, a dict from ``grad_buffers``, zeroed first unless
        ``zero`` is False).  ``stages``: HM_BWD_* bits to run (0 = all).
        With ``overlap`` (default ``self.overlap``) the blend replay and the
        projection gradients run on a high-priority side stream while the
        gradient zeroing and the texel gradients run on the current stream
        (the replay writes only its scratch; the projection gradients wait
        for the zeroing), and the streams join at the end.
        ``dL_dmesh`` (planar like ``rgb``): the gradient of a loss on the mesh
        colour itself, added to what the texels receive through I_h."""
        want_tex = tex_grad and self.has_mesh
        if (self.overlap if overlap is None else overlap) and want_tex and stages == 0:
            g = out if out is not None else self.grad_buffers(mesh.texture.shape[:2])
            main = torch.cuda.current_stream(self.device)
            hi = self._bin_stream()
            hi.wait_stream(main)
            with torch.cuda.stream(hi):          # the blend replay writes only its scratch
                self._backward_call(means, scales, quats, opacity, sh, dL_drgb, dL_dT, mesh, g,
                                    lib.HM_BWD_BLEND)
            if out is not None and zero:         # zeroed beside the replay
                for v in g.values():
                    v.zero_()
            zeroed = torch.cuda.Event()
            zeroed.record(main)
            self._backward_call(means, scales, quats, opacity, sh, dL_drgb, dL_dT, mesh, g,
                                lib.HM_BWD_TEXTURE, dL_dmesh)
            hi.wait_event(zeroed)
            with torch.cuda.stream(hi):
                self._backward_call(means, scales, quats, opacity, sh, dL_drgb, dL_dT, mesh, g,
                                    lib.HM_BWD_PROJECT)
            main.wait_stream(hi)
            return g
        if out is None:
            g = self.grad_buffers(mesh.texture.shape[:2] if want_tex else None)
        else:
            g = out
            if zero:
                for v in g.values():
                    v.zero_()
        self._backward_call(means, scales, quats, opacity, sh, dL_drgb, dL_dT, mesh if want_tex else None,
                            g, stages, dL_dmesh)
        return g

    def _backward_call(self, means, scales, quats, opacity, sh, dL_drgb, dL_dT, mesh, g, stages,
                       dL_dmesh=None):
        """One hm_blend_backward call on the current stream (texel gradients
        when ``mesh`` is given and ``g`` holds a texture buffer)."""
        if self.bwd_ws is None:
            self.bwd_ws = torch.empty(lib.hm_blend_backward_workspace_size(self.V, self.n),
                                      dtype=torch.uint8, device=self.device)
        d_tex = None
        tw = th = 0
        if mesh is not None and self.has_mesh and "texture" in g:
            th, tw = mesh.texture.shape[:2]
            d_tex = g["texture"]
        self.opt.bwd_stages = int(stages)
        lib.check(lib.hm_blend_backward(
            self.cams, self.n, means, scales, quats, opacity, sh, self.sh_degree, self.sh_format,
            self.records, self.pair_vals, self.ranges,
            self.mesh_depth if self.has_mesh else None, self.mesh_rgb if self.has_mesh else None,
            self.uv if self.has_mesh else None, tw, th, self.opt, self.T, self.last_idx,
            dL_drgb.contiguous(), None if dL_dT is None else dL_dT.contiguous(),
            g["means"], g["scales"], g["quats"], g["opacity"], g["sh"], d_tex, self.status_word,
            self.bwd_ws, self.bwd_ws.numel(), _stream(),
            dL_dmesh=None if (dL_dmesh is None or d_tex is None) else dL_dmesh.contiguous(),
            filter_3d=self.filter_3d),
            "hm_blend_backward")

    # -- the joint-optimisation loss ------------------------------------------------
    def loss(self, target: torch.Tensor, params=None, texture_loss: bool = True):
        """The joint loss of the last frame against ``target`` (planar like
        ``rgb``; float32 in [0, 1], or uint8 codes read as code / 255 by
        hm_hybrid_loss_u8) by hm_hybrid_loss: returns (terms, dL/drgb, dL/dmesh) with
        terms = device float64 [L1, mean SSIM, L_t, L] and dL/dmesh None
        without a mesh or with ``texture_loss`` off.  Pass both gradients to
        ``backward`` (``dL_drgb`` and ``dL_dmesh``)."""
        d = self.device
        if getattr(self, "_loss_ws", None) is None:
            self._loss_ws = torch.empty(lib.hm_hybrid_loss_workspace_size(self.cams), dtype=torch.uint8,
                                        device=d)
            self._loss_out = torch.empty(4, dtype=torch.float64, device=d)
            self._dI = torch.empty(3 * self.npix, dtype=torch.float32, device=d)
            self._dM = torch.empty(3 * self.npix, dtype=torch.float32, device=d) if self.has_mesh else None
        p = params if params is not None else lib.loss_params()
        use_mesh = self.has_mesh and texture_loss
        if target.dtype == torch.uint8:
            fn, name = lib.hm_hybrid_loss_u8, "hm_hybrid_loss_u8"
        elif target.dtype == torch.float32:
            fn, name = lib.hm_hybrid_loss, "hm_hybrid_loss"
        else:
            raise ValueError("target: uint8 or float32")
        lib.check(fn(self.cams, self.rgb, target.contiguous(),
                     self.mesh_rgb if use_mesh else None, self.T if use_mesh else None,
                     self.mesh_depth if use_mesh else None, p, self._loss_out, self._dI,
                     self._dM if use_mesh else None, self._loss_ws, self._loss_ws.numel(),
                     _stream()), name)
        return self._loss_out, self._dI, (self._dM if use_mesh else None)

    # -- views of the outputs -------------------------------------------------------
    def image(self, k: int, which: str = "rgb") -> torch.Tensor:
        w, h = self.sizes[k]
        a, b = int(self.pix_off[k]), int(self.pix_off[k + 1])
        if which == "rgb":
            return self.rgb[3 * a:3 * b].view(3, h, w)
        if which == "mesh_rgb":
            return self.mesh_rgb[3 * a:3 * b].view(3, h, w)
        if which == "uv":
            return self.uv[2 * a:2 * b].view(2, h, w)
        return getattr(self, which)[a:b].view(h, w)

    def records_view(self) -> torch.Tensor:
        return self.records[: self.V * self.n * 12].view(self.V * self.n, 12)


class HybridRender(torch.autograd.Function):
    """(means, scales, quats, opacity, sh[, texture]) -> (rgb, T) over all
    cameras of ``renderer`` (flat, as ``Renderer.rgb`` / ``Renderer.T``).
    The texture gets a gradient when it is float32 and requires grad."""

    @staticmethod
    def forward(ctx, renderer: Renderer, mesh: Optional[MeshInput], means, scales, quats, opacity,
                sh, texture=None):
        if mesh is not None and texture is not None:
            mesh = MeshInput(mesh.verts, mesh.uvs, mesh.faces, texture)
        means, scales, opacity = means.contiguous(), scales.contiguous(), opacity.contiguous()
        quats, sh = quats.contiguous(), sh.contiguous()
        renderer.render(means, scales, quats, opacity, sh, mesh)
        ctx.renderer = renderer
        ctx.mesh = mesh
        ctx.tex_grad = texture is not None and texture.requires_grad
        ctx.save_for_backward(means, scales, quats, opacity, sh)
        return renderer.rgb.clone(), renderer.T.clone()

    @staticmethod
    def backward(ctx, g_rgb, g_T):
        means, scales, quats, opacity, sh = ctx.saved_tensors
        r: Renderer = ctx.renderer
        g = r.backward(means, scales, quats, opacity, sh, g_rgb if g_rgb is not None else torch.zeros_like(r.rgb),
                       g_T, mesh=ctx.mesh, tex_grad=ctx.tex_grad)
        d_sh = g["sh"].to(sh.dtype) if sh.dtype != torch.float32 else g["sh"]
        return (None, None, g["means"], g["scales"], g["quats"], g["opacity"], d_sh,
                g.get("texture") if ctx.tex_grad else None)


class GraphStep:
    """One frame of a ``Renderer`` -- the forward stages and, when an upstream
    gradient is given, the backward pass into ``grads`` -- captured once in a
    CUDA graph and replayed with one launch call.

    A replay re-reads the current contents of the parameter tensors, the mesh
    and the upstream gradients, so callers update those in place between
    replays (the renderer's outputs and ``grads`` are overwritten each time).
    The capture follows an eager frame that settles the pair and work-item
    capacities; ``replay(check=True)`` synchronises, and on a capacity
    overflow grows the buffers eagerly and captures again.

    With a ``target`` (planar like ``rgb``; float32 in [0, 1], or uint8
    codes, which the loss kernels read as code / 255) the graph also
    evaluates the joint loss (hm_hybrid_loss with ``loss_params``) and
    back-propagates its
    gradient; ``loss_terms`` is then the device float64 [L1, mean SSIM,
    L_t, L] of the last replay.  With ``loss_host`` (a pinned float64 [4]
    host tensor) the replay also copies the loss terms there, as the graph's
    last operation: no separate read-back after each replay.
    """

    def __init__(self, renderer: Renderer, params, mesh: Optional[MeshInput] = None,
                 dL_drgb: Optional[torch.Tensor] = None, dL_dT: Optional[torch.Tensor] = None,
                 grads=None, tex_grad: bool = False, target: Optional[torch.Tensor] = None,
                 loss_params=None, loss_host: Optional[torch.Tensor] = None):
        self.r = renderer
        self.params = tuple(params)
        self.mesh = mesh
        self.dI, self.dT = dL_drgb, dL_dT
        if target is not None and dL_drgb is not None:
            raise ValueError("give either an upstream gradient or a target, not both")
        self.target = target
        if target is not None:
            if target.numel() != 3 * renderer.npix or not target.is_contiguous():
                raise ValueError("target: a contiguous planar image of every camera")
            if target.dtype not in (torch.uint8, torch.float32):
                raise ValueError("target: uint8 or float32")
        self.loss_params = loss_params if loss_params is not None else lib.loss_params()
        self.loss_terms = None
        if loss_host is not None:
            if target is None:
                raise ValueError("loss_host needs a target (the loss is evaluated in the graph)")
            if loss_host.device.type != "cpu" or not loss_host.is_pinned() or loss_host.dtype != torch.float64 \
                    or loss_host.numel() != 4:
                raise ValueError("loss_host: a pinned float64 host tensor of 4 elements")
        self.loss_host = loss_host
        self.tex_grad = bool(tex_grad and renderer.has_mesh)
        self.grads = grads
        if (self.dI is not None or target is not None) and self.grads is None:
            self.grads = renderer.grad_buffers(mesh.texture.shape[:2] if self.tex_grad else None)
        self.graph = None
        self.capture()

    def _body(self):
        r = self.r
        r.forward(*self.params, self.mesh, overlap=True)
        dI, dM = self.dI, None
        if self.target is not None:
            self.loss_terms, dI, dM = r.loss(self.target, self.loss_params,
                                             texture_loss=self.tex_grad and self.loss_params.lambda_t > 0)
        if dI is not None:
            r.backward(*self.params, dI, self.dT, mesh=self.mesh, tex_grad=self.tex_grad,
                       out=self.grads, zero=True, overlap=True, dL_dmesh=dM)
        if self.loss_host is not None:
            self.loss_host.copy_(self.loss_terms, non_blocking=True)

    def capture(self):
        r = self.r
        r.render(*self.params, self.mesh, overlap=True)   # settles the capacities the graph needs
        side = torch.cuda.Stream(device=r.device)
        side.wait_stream(torch.cuda.current_stream(r.device))
        with torch.cuda.stream(side):                    # lazy workspaces, first-call set-up
            self._body()
        torch.cuda.current_stream(r.device).wait_stream(side)
        torch.cuda.synchronize(r.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._body()
        self.graph = g
        return self

    def replay(self, check: bool = False):
        self.graph.replay()
        if check:
            st, npairs, nitems = self.r.status()
            lib.check_device_status(st)
            if st & lib.HM_DEV_CAPACITY:
                self.capture()                            # grows the buffers, then re-captures
                self.graph.replay()
        return self


class ChunkedRenderer:
    """Many cameras rendered ``chunk`` at a time through one renderer's
    scratch: records, sorted per-tile lists and workspaces exist for one
    chunk only.  The per-pixel outputs of every camera are kept (they are the
    backward pass's inputs); the backward pass re-projects each chunk and
    recomputes its sorted lists instead of storing them -- bit-identical
    lists, since the projection and the sort are deterministic.

    Chunks of different camera sizes get a renderer each (one per distinct
    size pattern).
    """

    def __init__(self, cams, n: int, sh_degree: int, *, chunk: int, device="cuda", **kw):
        self.cam_list = list(cams)
        self.V = len(self.cam_list)
        self.chunk = max(1, int(chunk))
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.K = (self.sh_degree + 1) ** 2
        self.kw = dict(kw)
        self.device = torch.device(device)
        self.sizes = [(int(c.width), int(c.height)) for c in self.cam_list]
        self.pix_off = np.concatenate([[0], np.cumsum([w * h for w, h in self.sizes])]).astype(np.int64)
        self.npix = int(self.pix_off[-1])
        tw, th = kw.get("tile", (16, 16))
        tiles = [((w + tw - 1) // tw) * ((h + th - 1) // th) for w, h in self.sizes]
        self.tile_off = np.concatenate([[0], np.cumsum(tiles)]).astype(np.int64)
        self.has_mesh = kw.get("n_faces", 0) > 0 or kw.get("tex_shape") is not None
        d = self.device
        fields = Renderer.PIXEL_FIELDS + (Renderer.MESH_FIELDS if self.has_mesh else ())
        for name, per, dt in fields:
            setattr(self, name, torch.empty(per * self.npix, dtype=dt, device=d))
        self.tile_max = torch.empty(int(self.tile_off[-1]), dtype=torch.float32, device=d) if self.has_mesh else None
        self.chunks = [list(range(i, min(i + self.chunk, self.V))) for i in range(0, self.V, self.chunk)]
        self._renderers = {}
        self.filter_3d: Optional[torch.Tensor] = None

    def set_filter_3d(self, v: Optional[torch.Tensor]):
        """Mip-Splatting's 3D smoothing variance for every chunk's projection
        (compute it over all cameras, e.g. with ``Renderer.mip_filter_3d``)."""
        self.filter_3d = v
        for r in self._renderers.values():
            r.set_filter_3d(v)

    def _bufs(self, idx):
        a, b = int(self.pix_off[idx[0]]), int(self.pix_off[idx[-1] + 1])
        out = {}
        fields = Renderer.PIXEL_FIELDS + (Renderer.MESH_FIELDS if self.has_mesh else ())
        for name, per, _ in fields:
            out[name] = getattr(self, name)[per * a:per * b]
        if self.has_mesh:
            out["tile_max"] = self.tile_max[int(self.tile_off[idx[0]]):int(self.tile_off[idx[-1] + 1])]
        return out

    def renderer(self, ci: int) -> Renderer:
        """The renderer set up for chunk ``ci`` (cameras and output slices)."""
        idx = self.chunks[ci]
        cams = [self.cam_list[k] for k in idx]
        key = tuple(self.sizes[k] for k in idx)
        r = self._renderers.get(key)
        if r is None:
            r = Renderer(cams, self.n, self.sh_degree, pixel_buffers=self._bufs(idx), device=self.device,
                         **self.kw)
            r.set_filter_3d(self.filter_3d)
            self._renderers[key] = r
        else:
            r.retarget(cams, self._bufs(idx))
        return r

    def render(self, means, scales, quats, opacity, sh, mesh: Optional[MeshInput] = None):
        """Forward pass of every chunk (capacity checks synchronise per chunk)."""
        for ci in range(len(self.chunks)):
            self.renderer(ci).render(means, scales, quats, opacity, sh, mesh)
        return self

    def forward(self, means, scales, quats, opacity, sh, mesh: Optional[MeshInput] = None):
        """Forward pass of every chunk, asynchronously (capacities as settled
        by an earlier ``render``)."""
        for ci in range(len(self.chunks)):
            self.renderer(ci).forward(means, scales, quats, opacity, sh, mesh)
        return self

    def status(self, check: bool = False):
        """OR of the chunk renderers' status bits -- synchronises.  With
        ``check``, raises on HM_DEV_TIMEOUT and HM_DEV_BAD_INDEX."""
        st = 0
        for r in self._renderers.values():
            st |= r.status()[0]
        return lib.check_device_status(st) if check else st

    def grad_buffers(self, tex_shape=None):
        d = self.device
        g = dict(means=torch.zeros(self.n, 3, device=d), scales=torch.zeros(self.n, 3, device=d),
                 quats=torch.zeros(self.n, 4, device=d), opacity=torch.zeros(self.n, device=d),
                 sh=torch.zeros(self.n, self.K, 3, device=d))
        if tex_shape is not None:
            g["texture"] = torch.zeros(tex_shape[0], tex_shape[1], 3, device=d)
        return g

    def backward(self, means, scales, quats, opacity, sh, dL_drgb, dL_dT=None,
                 mesh: Optional[MeshInput] = None, tex_grad: bool = False, out=None, zero: bool = True):
        """Gradients of the last forward: per chunk, re-project and re-sort
        (the lists are recomputed, not stored), then the backward kernels,
        accumulating into one set of gradient buffers."""
        want_tex = tex_grad and self.has_mesh
        g = out if out is not None else self.grad_buffers(mesh.texture.shape[:2] if want_tex else None)
        if out is not None and zero:
            for v in g.values():
                v.zero_()
        for ci, idx in enumerate(self.chunks):
            r = self.renderer(ci)
            a, b = int(self.pix_off[idx[0]]), int(self.pix_off[idx[-1] + 1])
            r.project(means, scales, quats, opacity, sh)
            r.bin_sort()
            r.backward(means, scales, quats, opacity, sh, dL_drgb[3 * a:3 * b],
                       None if dL_dT is None else dL_dT[a:b], mesh=mesh, tex_grad=want_tex, out=g,
                       zero=False)
        return g
