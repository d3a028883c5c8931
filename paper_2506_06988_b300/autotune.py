"""Tile-shape, staging-batch and launch-mode autotuner for the renderer.

The image does not depend on either choice (the 3-sigma test is per pixel,
so the per-pixel candidate set is the same for every tile shape, and the
staging batch only changes how the depth-sorted list is walked), but the
cost does: small tiles duplicate more (Gaussian, tile) pairs in the sort,
large tiles make more pixels walk entries that miss them, and the batch
trades shared-memory rounds against entries staged past a tile's early
exit.  The launch mode (one CTA per tile, or a persistent grid of resident
CTAs claiming (view, tile) work from a counter) does not change the result
either.  ``tune`` times the whole frame (forward, and backward when an
upstream gradient is given) for every valid (tile, batch, launch) on the
caller's own cameras and scene, with CUDA events on the current stream, and
returns the fastest with its renderer ready to use.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

from .render import MeshInput, Renderer

__all__ = ["TILES", "BATCHES", "LAUNCHES", "TuneResult", "tune"]

TILES = ((16, 16), (32, 8), (8, 8))
BATCHES = (32, 64, 128, None)          # None: one tile's worth of pixels
LAUNCHES = (False, True)               # persistent work-queue launch of the blend kernels


@dataclass
class TuneResult:
    tile: tuple
    batch: int
    ms: float
    renderer: Renderer
    table: list = field(default_factory=list)   # (tile, batch, persistent, ms per frame)
    persistent: bool = False


def _time_frames(r: Renderer, params, mesh, dI, grads, tex_grad, warmup, iters):
    s = torch.cuda.current_stream(r.device)
    for _ in range(warmup):
        r.forward(*params, mesh)
        if dI is not None:
            r.backward(*params, dI, None, mesh=mesh, tex_grad=tex_grad, out=grads, zero=True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for _ in range(iters):
        r.forward(*params, mesh)
        if dI is not None:
            r.backward(*params, dI, None, mesh=mesh, tex_grad=tex_grad, out=grads, zero=True)
    t1.record(s)
    t1.synchronize()
    return t0.elapsed_time(t1) / iters


def tune(cams, n: int, sh_degree: int, params, mesh: Optional[MeshInput] = None, *,
         dL_drgb: Optional[torch.Tensor] = None, tex_grad: bool = False,
         tiles: Sequence = TILES, batches: Sequence = BATCHES, launches: Sequence = LAUNCHES,
         warmup: int = 2, iters: int = 5, **renderer_kw) -> TuneResult:
    """Time every valid (tile, batch, launch) and return the fastest.

    ``params`` = (means, scales, quats, opacity, sh) on the device; the
    remaining keyword arguments go to ``Renderer`` (sh_f16, n_verts, n_faces,
    tex_shape, bg, ...).  Batches above a tile's pixel count are skipped.
    """
    best = None
    table = []
    for tile in tiles:
        r = Renderer(cams, n, sh_degree, tile=tuple(tile), **renderer_kw)
        r.render(*params, mesh)                        # settles the capacities
        grads = None
        if dL_drgb is not None:
            grads = r.grad_buffers(mesh.texture.shape[:2] if (tex_grad and mesh is not None) else None)
        npx = tile[0] * tile[1]
        tried = set()
        for b in batches:
            bb = npx if b is None else int(b)
            if bb > npx or bb in tried:
                continue
            tried.add(bb)
            r.opt.batch = bb
            for pers in launches:
                r.opt.persistent = int(bool(pers))
                ms = _time_frames(r, params, mesh, dL_drgb, grads, tex_grad, warmup, iters)
                table.append((tuple(tile), bb, bool(pers), ms))
                if best is None or ms < best[3]:
                    best = (tuple(tile), bb, bool(pers), ms)
        del r, grads
    tile, batch, pers, ms = best
    r = Renderer(cams, n, sh_degree, tile=tile, batch=batch, persistent=pers, **renderer_kw)
    r.render(*params, mesh)
    return TuneResult(tile=tile, batch=batch, ms=ms, renderer=r, table=table, persistent=pers)
