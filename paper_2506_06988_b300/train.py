"""One joint-optimisation step of the hybrid representation (Sec. 3.4) as a
single CUDA graph.

The step trains the 3DGS parameterisation -- means, log-scales, quaternions,
opacity logits, SH coefficients -- and the FP32 texels of the mesh:

  activations (hm_activate)  ->  hybrid render (mesh pass, projection,
  binning, blend)  ->  joint loss (hm_hybrid_loss: Eq. 3 + lambda_t L_t of
  Eq. 5/7)  ->  gradients (texels, blend, projection; hm_blend_backward)
  ->  chain rule through the activations (hm_activate_backward)  ->  Adam on
  the six parameter groups (hm_adam_advance + hm_adam_update_dev).

Everything is a kernel of the library on one stream (side streams inside);
the graph is captured once and replayed per step.  The Adam step counter and
bias corrections live in device memory, and every update is skipped when a
stage of the step reported an error in the renderer's status word (e.g. a
pair-capacity overflow), so ``step(check=True)`` can grow the buffers,
capture again and redo the step with the parameters untouched.

lambda_t follows the warm-up schedule (Algorithm 1) through
``set_texture_loss_weight``, which captures again when the weight changes.
"""
from __future__ import annotations

from typing import Dict, Optional

import torch

from . import lib
from .render import MeshInput, Renderer

GROUPS = ("means", "log_scales", "quats", "logit", "sh", "texture")


class JointTrainStep:
    """``params``: dict of device float32 tensors means [n,3], log_scales
    [n,3], quats [n,4], logit [n], sh [n,K,3], updated in place; ``mesh``
    with a float32 texture (the texel parameter, updated in place);
    ``target``: planar RGB of every camera, like ``Renderer.rgb``."""

    def __init__(self, renderer: Renderer, params: Dict[str, torch.Tensor], mesh: MeshInput,
                 target: torch.Tensor, *, lrs: Optional[Dict[str, float]] = None, betas=(0.9, 0.999),
                 eps: float = 1e-15, lambda_ssim: float = 0.2, lambda_t: float = 0.0):
        r = renderer
        if mesh.texture.dtype != torch.float32:
            raise ValueError("the texel parameter must be float32")
        self.r = r
        self.p = {k: params[k] for k in GROUPS[:-1]}
        self.p["texture"] = mesh.texture
        for k, v in self.p.items():
            if not v.is_contiguous() or v.dtype != torch.float32:
                raise ValueError(f"{k}: need a contiguous float32 tensor")
        self.mesh = mesh
        self.target = target.contiguous()
        d = r.device
        n = r.n
        self.scales = torch.empty(n, 3, dtype=torch.float32, device=d)
        self.opacity = torch.empty(n, dtype=torch.float32, device=d)
        self.grads = r.grad_buffers(tuple(mesh.texture.shape[:2]))
        self.d_log_s = torch.zeros(n, 3, dtype=torch.float32, device=d)
        self.d_logit = torch.zeros(n, dtype=torch.float32, device=d)
        default_lr = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, logit=5e-2, sh=2.5e-3, texture=1e-2)
        self.lrs = dict(default_lr, **(lrs or {}))
        self.betas, self.eps = (float(betas[0]), float(betas[1])), float(eps)
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.d_step = torch.zeros(1, dtype=torch.int32, device=d)
        self.d_rc = torch.ones(2, dtype=torch.float32, device=d)
        self.lambda_ssim = float(lambda_ssim)
        self.lambda_t = float(lambda_t)
        self.terms = None
        self.graph = None
        self.capture()

    # -- the step --------------------------------------------------------------------
    def _grad_of(self, k):
        return dict(means=self.grads["means"], log_scales=self.d_log_s, quats=self.grads["quats"],
                    logit=self.d_logit, sh=self.grads["sh"], texture=self.grads["texture"])[k]

    def _body(self, update: bool = True):
        r, p = self.r, self.p
        s = torch.cuda.current_stream(r.device).cuda_stream
        lib.check(lib.hm_activate(r.n, p["log_scales"], p["logit"], self.scales, self.opacity, s), "hm_activate")
        P = (p["means"], self.scales, p["quats"], self.opacity, p["sh"])
        r.forward(*P, self.mesh, overlap=True)
        lp = lib.loss_params(lambda_ssim=self.lambda_ssim, lambda_t=self.lambda_t)
        terms, dI, dM = r.loss(self.target, lp, texture_loss=self.lambda_t > 0)
        r.backward(*P, dI, None, mesh=self.mesh, tex_grad=True, out=self.grads, zero=True, overlap=True,
                   dL_dmesh=dM)
        s = torch.cuda.current_stream(r.device).cuda_stream
        lib.check(lib.hm_activate_backward(r.n, self.scales, self.opacity, self.grads["scales"],
                                           self.grads["opacity"], self.d_log_s, self.d_logit, s),
                  "hm_activate_backward")
        self.terms = terms
        if not update:
            return
        b1, b2 = self.betas
        lib.check(lib.hm_adam_advance(self.d_step, b1, b2, self.d_rc, r.status_word, s), "hm_adam_advance")
        for k in GROUPS:
            lib.check(lib.hm_adam_update_dev(p[k], self._grad_of(k), self.m[k], self.v[k], p[k].numel(),
                                             self.lrs[k], b1, b2, self.eps, self.d_rc, r.status_word, s),
                      "hm_adam_update_dev")

    def capture(self):
        r, p = self.r, self.p
        # settle the pair / work-item capacities with the current parameters
        s = torch.cuda.current_stream(r.device).cuda_stream
        lib.check(lib.hm_activate(r.n, p["log_scales"], p["logit"], self.scales, self.opacity, s), "hm_activate")
        r.render(p["means"], self.scales, p["quats"], self.opacity, p["sh"], self.mesh, overlap=True)
        side = torch.cuda.Stream(device=r.device)
        side.wait_stream(torch.cuda.current_stream(r.device))
        with torch.cuda.stream(side):                    # lazy workspaces; no parameter update
            self._body(update=False)
        torch.cuda.current_stream(r.device).wait_stream(side)
        torch.cuda.synchronize(r.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._body()
        self.graph = g
        return self

    def step(self, check: bool = False) -> torch.Tensor:
        """One optimisation step; returns the device float64 loss terms
        [L1, mean SSIM, L_t, L] of the render before the update.  With
        ``check`` the status is read (a synchronisation): after a capacity
        overflow (no parameter was updated) the buffers grow, the step is
        captured again and redone."""
        self.graph.replay()
        if check:
            st, _, _ = self.r.status()
            lib.check_device_status(st)
            if st & lib.HM_DEV_CAPACITY:
                self.capture()
                self.graph.replay()
        return self.terms

    def set_texture_loss_weight(self, lambda_t: float):
        """Change lambda_t (Algorithm 1's schedule); captures again if it changed."""
        if float(lambda_t) != self.lambda_t:
            self.lambda_t = float(lambda_t)
            self.capture()

    @property
    def iteration(self) -> int:
        return int(self.d_step.item())
