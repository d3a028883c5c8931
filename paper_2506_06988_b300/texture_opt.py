"""Texture optimisation from images alone: the texture-map initialisation
that precedes the joint optimisation (Sec. 3.3, Algorithm 1 stage 1), where
the texels of the pruned mesh are fitted to the training images through a
differentiable rasteriser.

Each step renders the mesh alone for every camera (hm_rasterize_mesh, then
hm_blend_forward with no Gaussians, so I = I_m where a triangle covers the
pixel and the background elsewhere), evaluates the photometric loss of Eq. 3
(hm_hybrid_loss: 0.8 L1 + 0.2 D-SSIM), takes the texel gradient
(hm_blend_backward, texture part) and applies Adam to the texels
(hm_adam_advance + hm_adam_update_dev: the step counter and the bias
corrections live in device memory, and the update is skipped when a stage
reported an error).  All of it runs in the library's kernels on the current
stream; the host only sequences the calls, or replays them as one CUDA graph
after ``capture()``.  The mesh is fixed, so its work-item capacity is settled
once by a checked render at construction.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import lib
from .render import MeshInput, Renderer


class TextureOptimizer:
    """Fits ``mesh``'s texture (copied to a float32 parameter, ``texture``)
    to ``targets`` (planar RGB per camera, concatenated like
    ``Renderer.rgb``)."""

    def __init__(self, cams, mesh: MeshInput, targets: torch.Tensor, *, lr: float = 1e-2,
                 betas=(0.9, 0.999), eps: float = 1e-8, lambda_ssim: float = 0.2, bg=(0.0, 0.0, 0.0),
                 tile=(16, 16), device="cuda"):
        d = torch.device(device)
        tex = mesh.texture
        if tex.dtype != torch.float32:
            tex = tex.to(torch.float32) / 255.0
        self.texture = tex.to(d).contiguous().clone()
        self.mesh = MeshInput(mesh.verts, mesh.uvs, mesh.faces, self.texture)
        self.r = Renderer(cams, 0, 0, n_verts=int(mesh.verts.shape[0]), n_faces=int(mesh.faces.shape[0]),
                          tex_shape=tuple(self.texture.shape), bg=bg, tile=tile, device=d)
        if targets.numel() != 3 * self.r.npix:
            raise ValueError(f"targets: need {3 * self.r.npix} values (planar RGB of every camera)")
        self.targets = targets.to(d, torch.float32).contiguous()
        self.lr, self.betas, self.eps = float(lr), (float(betas[0]), float(betas[1])), float(eps)
        self.m = torch.zeros_like(self.texture)
        self.v = torch.zeros_like(self.texture)
        self.d_step = torch.zeros(1, dtype=torch.int32, device=d)
        self.d_rc = torch.ones(2, dtype=torch.float32, device=d)
        self.loss_params = lib.loss_params(lambda_ssim=lambda_ssim, lambda_t=0.0)
        self.grads = self.r.grad_buffers(tuple(self.texture.shape[:2]))
        f32 = dict(dtype=torch.float32, device=d)
        self._none = (torch.empty(0, 3, **f32), torch.empty(0, 3, **f32), torch.empty(0, 4, **f32),
                      torch.empty(0, **f32), torch.empty(0, 1, 3, **f32))
        self.graph = None
        self.r.render(*self._none, self.mesh)        # settles the mesh work-item capacity

    def render(self) -> torch.Tensor:
        """The mesh render of every camera with the current texels."""
        self.r.forward(*self._none, self.mesh)
        return self.r.rgb

    def _body(self, update: bool = True):
        self.render()
        terms, dI, _ = self.r.loss(self.targets, self.loss_params, texture_loss=False)
        self.r.backward(*self._none, dI, None, mesh=self.mesh, tex_grad=True, out=self.grads,
                        stages=lib.HM_BWD_TEXTURE)
        self.terms = terms
        if not update:
            return
        s = torch.cuda.current_stream(self.texture.device).cuda_stream
        b1, b2 = self.betas
        lib.check(lib.hm_adam_advance(self.d_step, b1, b2, self.d_rc, self.r.status_word, s), "hm_adam_advance")
        lib.check(lib.hm_adam_update_dev(self.texture, self.grads["texture"], self.m, self.v, self.texture.numel(),
                                         self.lr, b1, b2, self.eps, self.d_rc, self.r.status_word, s),
                  "hm_adam_update_dev")

    def capture(self):
        """Capture one step as a CUDA graph; ``step`` then replays it."""
        d = self.texture.device
        side = torch.cuda.Stream(device=d)
        side.wait_stream(torch.cuda.current_stream(d))
        with torch.cuda.stream(side):                    # lazy workspaces; no update
            self._body(update=False)
        torch.cuda.current_stream(d).wait_stream(side)
        torch.cuda.synchronize(d)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._body()
        self.graph = g
        return self

    def step(self, check: bool = False) -> torch.Tensor:
        """One optimisation step (the captured graph, if any); returns the
        device float64 loss terms [L1, mean SSIM, 0, L] of the render before
        the update.  With ``check`` the status word is read (a
        synchronisation) and an error raises (no texel was updated)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body()
        if check:
            st, _, _ = self.r.status()
            if st:
                raise lib.HmError(f"texture step: device status {st:#x} (the update was skipped)")
        return self.terms

    @property
    def t(self) -> int:
        """Steps taken (reads the device counter: a synchronisation)."""
        return int(self.d_step.item())

    def run(self, steps: int, log_every: Optional[int] = None):
        """``steps`` steps; returns the final loss terms (host floats)."""
        terms = None
        for k in range(steps):
            terms = self.step()
            if log_every and (k + 1) % log_every == 0:
                print(f"step {k + 1}: L = {float(terms[3]):.6f}")
        return [float(x) for x in terms.cpu()] if terms is not None else None
