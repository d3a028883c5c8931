"""Benchmark of the hybrid mesh-Gaussian renderer on B300.

Workload (N=1): the seeded indoor-room scene at 1920x1080 -- 8 camera poses,
300k Gaussians (SH degree 3), a 6x5x3 m room of ~50k triangles with 10%
pruned in clusters, 2048^2 RGB8 atlas.  A step is one pass of the whole hot
path over the 8 views: mesh rasterisation, projection, bin/sort, hybrid blend
(forward) and the backward pass (blend, texture and projection gradients)
for a fixed seeded upstream gradient dL/dI.  Metric: frames/s (views per
second) and Mpixel/s, forward+backward; the forward-only rate is reported
beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N>1) every rank renders its own block of 8 views of the same
room (weak scaling; no collective on the data path) and rank 0 prints the line with the
max-over-ranks time.  ``--impl reference`` times the CPU FP64 oracle (the
correctness reference; there is no other implementation of this path) on the
host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hybrid render frames/s & Mpixel/s at 1080p (fwd, fwd+bwd) and % of roofline"
UNIT = "frames/s"
WORKLOAD = ("indoor room 1920x1080 x 8 poses, 300k Gaussians SH3, 50k-triangle room mesh "
            "(10% pruned), 2048^2 RGB8 atlas; forward + backward")
# Work of the blend kernels per (pixel, Gaussian) pair, two counts:
# * the nominal count of the method's arithmetic per evaluated pair (inside
#   the 3-sigma ellipse): ~12 FP32 operations + 1 ex2 forward, ~40 + 1 ex2
#   backward, counted as FLOPs against the FP32 peak (an FMA as two);
# * the count read off the kernel sources (per evaluated pair forward, per
#   blended pair backward; an FMA as two, packed FP32x2 ops per pixel):
#   forward q 7 (dx, a dx^2 and 2b dx shared by the pixel pair), the 3-sigma,
#   alpha and T-stop compares 3, alpha 2 (o 2^q, min), T' 2, the alpha
#   select 1, weight 1, colour 6, T 2, mesh cut 1 = 25; backward (no dL/dT)
#   q 6 (the column part shared by four pixels), the 3-sigma and alpha
#   compares 2, alpha 2, the blended select 1, 1 - alpha 1, T_i 1, weight
#   1, colour partials 6, c - B 3, the dot with dL/dI 5, dL/dalpha 1, the
#   clamp test and select 2, dL/dq 1, gq dy 1, the moment sums 4, the colour
#   behind 6, the entry's horizontal adds and moment and dL/do products
#   shared by the lane's four pixels 3 = 46 (+ ex2 and rcp).
METHOD_FLOPS = {"blend_forward": 12, "blend_backward": 40}
SOURCE_FLOPS = {"blend_forward": 25, "blend_backward": 46}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) and warp
# instructions (smsp__inst_executed.sum) of one launch of each blend kernel,
# from an ncu capture of 3 of the 8 views (profiles/blend_*_kernel_room1080p_3views.md)
# with the sources the kernel was built from.  A full launch's figure is the
# capture scaled by the live workload: instructions by the kernel's units
# (evaluated pairs forward, blended pairs backward), traffic by pixels.  A
# figure is reported only while the sources hash to the recorded value.
KERNEL_SOURCES = {
    "blend_forward": ("blend_fwd.cu", "blend_common.cuh", "hm_internal.cuh", "tma.cuh"),
    "blend_backward": ("blend_bwd.cu", "blend_common.cuh", "hm_internal.cuh", "tma.cuh"),
    "texture_backward": ("blend_bwd.cu", "blend_common.cuh", "hm_internal.cuh", "tma.cuh"),
    "project_backward": ("blend_bwd.cu", "blend_common.cuh", "hm_internal.cuh", "sh.cuh", "tma.cuh"),
    "project": ("project.cu", "sh.cuh", "hm_internal.cuh"),
}
NCU_CAPTURE = {
    # stage: (warp instructions, DRAM bytes, units, unit kind, pixels, source hash)
    "blend_forward": (182_410_274, 219_468_288, 113_755_470, "evaluated_pairs", 3 * 1920 * 1080, "2be5ebbb112a845f"),
    "blend_backward": (256_249_321, 122_555_136, 110_624_405, "blended_pairs", 3 * 1920 * 1080, "e614eeda23b39bd3"),
}


def _source_hash(stage):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[stage]:
        with open(os.path.join(ROOT, "paper_2506_06988_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _captured(stage, tile, units, pixels):
    """(warp instructions, DRAM bytes) of one launch scaled from the
    committed capture, or (None, None) when the kernel's sources or tile
    shape differ from the captured ones."""
    if stage not in NCU_CAPTURE or tuple(tile) != (16, 16):
        return None, None
    inst, dram, cap_units, kind, cap_px, digest = NCU_CAPTURE[stage]
    if _source_hash(stage) != digest:
        return None, None
    return inst * units[kind] / cap_units, dram * pixels / cap_px


KERNELS_PER_STEP = {"rasterize_mesh": 6, "project": 1, "bin_sort": 9, "blend_forward": 1,
                    "texture_backward": 1, "blend_backward": 1, "project_backward": 1}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (read only)."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    """(rank, world, local rank, torch.distributed or None) from the torchrun
    environment; NCCL between the GPUs (HM_BENCH_BACKEND=gloo runs the same
    host logic on CPU processes, for tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = os.environ.get("HM_BENCH_BACKEND", "nccl")
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def _on_gpu(dist) -> bool:
    return dist is None or dist.get_backend() == "nccl"


def _max_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _on_gpu(dist) else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    import torch
    gpu = _on_gpu(dist) and torch.cuda.is_available()
    if gpu:
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    if gpu:
        torch.cuda.synchronize()


def view_block_scene(rank: int):
    """The headline scene with rank ``rank``'s own block of 8 poses of the
    same room (data parallel over views: no collective on the data path)."""
    from paper_2506_06988_b300 import scenes
    return scenes.config1_scene(view_block=rank)


# ----------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ----------------------------------------------------------------------------

def cpu_oracle_sample(scene, rows=8, crop=12, t_fixed=None):
    """Time the CPU FP64 oracle on a bounded sample of one 1080p view: the
    mesh pass and the blend over a band of `rows` full rows (exact grid
    prefilter), the projection of all Gaussians, and the FP64 gradient
    oracle (autograd) over a crop x crop pixel block.  The gradient run's
    per-frame part (the projection through autograd) is `t_fixed` seconds
    when given, else timed from a one-pixel run.  Returns seconds per full
    frame for forward and forward+backward."""
    import torch
    from oracle import oracle as O
    from oracle import torch_ref as TR

    cam = scene.cameras[0]
    W, H = cam.width, cam.height
    y0 = H // 2 - rows // 2
    t0 = time.perf_counter()
    pr = O.project(cam, scene.gaussians)
    t_proj = time.perf_counter() - t0
    pix = np.arange(y0 * W, (y0 + rows) * W, dtype=np.int64)
    t0 = time.perf_counter()
    mr = O.mesh_raster(cam, scene.mesh, bg=scene.bg, pix=pix)
    t_mesh = time.perf_counter() - t0
    full = O.empty_mesh_result(W * H, scene.bg)
    full.tri_id[pix], full.depth[pix] = mr.tri_id, mr.depth
    full.depth64[pix], full.depth_tol[pix], full.tri_margin[pix] = mr.depth64, mr.depth_tol, mr.tri_margin
    full.rgb[:, pix] = mr.rgb
    t0 = time.perf_counter()
    O.blend_grid(cam, pr, scene.gaussians.opacity, full, bg=scene.bg, rows=(y0, y0 + rows))
    t_blend = time.perf_counter() - t0
    fwd = t_proj + (t_mesh + t_blend) * (H / rows)
    # backward over a crop x crop block centred in the view (single view scene)
    cx0, cy0 = W // 2 - crop // 2, H // 2 - crop // 2
    cpix = np.array([(cy0 + j) * W + cx0 + i for j in range(crop) for i in range(crop)], np.int64)
    gI = np.random.default_rng(0).standard_normal((3, len(cpix)))
    sub = type(scene)(scene.name, scene.seed, scene.gaussians, scene.mesh, [cam], scene.bg)
    torch.set_num_threads(O.num_threads())
    # per-frame part (projection through autograd) from a 1-pixel run, per-pixel
    # part from the crop
    if t_fixed is None:
        t0 = time.perf_counter()
        TR.render_grad(sub, 0, gI[:, :1], pix=cpix[:1], chunk=8)
        t_fixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    TR.render_grad(sub, 0, gI, pix=cpix, chunk=8)
    t_bwd = time.perf_counter() - t0
    bwd = t_fixed + max(t_bwd - t_fixed, 0.0) * (W * H) / len(cpix)
    return fwd, fwd + bwd, {"rows": rows, "crop": crop, "t_proj": t_proj, "t_mesh": t_mesh,
                            "t_blend": t_blend, "t_bwd_crop": t_bwd, "t_bwd_fixed": t_fixed}


def cpu_oracle_small():
    """The oracle on the whole small case (one 128x128 view, 2000 Gaussians
    SH0, a textured quad): the forward frame and the FP64 autograd gradient
    of every pixel, unsampled."""
    import torch
    from oracle import oracle as O
    from oracle import torch_ref as TR
    from paper_2506_06988_b300 import scenes
    s = scenes.config0_scene()
    cam = s.cameras[0]
    torch.set_num_threads(O.num_threads())
    t0 = time.perf_counter()
    O.render(s)
    fwd = time.perf_counter() - t0
    gI = np.random.default_rng(0).standard_normal((3, cam.width * cam.height))
    t0 = time.perf_counter()
    TR.render_grad(s, 0, gI, chunk=1024)
    bwd = time.perf_counter() - t0
    return {"workload": "128x128 view, 2000 Gaussians SH0, textured quad (the whole frame)",
            "forward_frames_per_s": 1.0 / fwd, "frames_per_s": 1.0 / (fwd + bwd), "cores": O.num_threads()}


def fixed_grad_cost(scene):
    """Seconds of the FP64 gradient oracle's per-frame part on view 0 of
    `scene`: a one-pixel run, median of three after a warm-up run."""
    import torch
    from oracle import oracle as O
    from oracle import torch_ref as TR
    cam = scene.cameras[0]
    W, H = cam.width, cam.height
    pix = np.array([(H // 2) * W + W // 2], np.int64)
    gI = np.ones((3, 1))
    sub = type(scene)(scene.name, scene.seed, scene.gaussians, scene.mesh, [cam], scene.bg)
    torch.set_num_threads(O.num_threads())
    ts = []
    for _ in range(4):
        t0 = time.perf_counter()
        TR.render_grad(sub, 0, gI, pix=pix, chunk=8)
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts[1:]))


def run_reference(args):
    rank, ws, _, dist = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2506_06988_b300 import scenes
    scene = scenes.config1_scene()
    steps, warm = args.steps, args.warmup
    # the gradient oracle's per-frame part (projection through autograd),
    # timed once (median of three one-pixel runs after a warm-up one), so
    # that each step's 8 x 8 block measures the per-pixel part
    t_fixed = fixed_grad_cost(scene)
    times = []
    info = {}
    for i in range(warm + steps):
        fwd, fb, info = cpu_oracle_sample(scene, rows=4, crop=8, t_fixed=t_fixed)
        if i >= warm:
            times.append(fb)
    sec_per_frame = float(np.mean(times))
    value = 1.0 / sec_per_frame
    mpx = value * 1920 * 1080 / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 8 * sec_per_frame * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "mpixel_per_s": mpx,
            "config": {"workload": WORKLOAD, "views": 8, "width": 1920, "height": 1080, "gaussians": 300000,
                       "seed": 1, "sh_degree": 3},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "each step: oracle forward over 4 rows of one 1080p view "
                                       "(+ full projection) and FP64 autograd backward over an 8x8 "
                                       "block, scaled to a full frame (the backward's per-frame part "
                                       f"timed once: {t_fixed:.2f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# CUDA path
# ----------------------------------------------------------------------------

def run_ours(args):
    import torch
    from paper_2506_06988_b300 import lib, scenes
    from paper_2506_06988_b300.render import HybridRender, MeshInput, Renderer

    rank, world, local, dist = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lib.load()
    scene = view_block_scene(rank)
    scene.cameras = scene.cameras[:args.views]
    g = scene.gaussians
    tile = tuple(int(x) for x in args.tile.split("x"))
    V = len(scene.cameras)
    r = Renderer(scene.cameras, g.n, g.sh_degree, n_verts=len(scene.mesh.verts),
                 n_faces=len(scene.mesh.faces), tex_shape=scene.mesh.texture.shape, tile=tile,
                 batch=args.batch, bg=tuple(scene.bg), device=dev)
    P = {k: torch.as_tensor(getattr(g, k), device=dev).contiguous()
         for k in ("means", "scales", "quats", "opacity", "sh")}
    mesh = MeshInput.from_numpy(scene.mesh, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    dI = torch.randn(3 * r.npix, device=dev, generator=gen) * 1e-3
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)   # settles capacities
    grads = r.grad_buffers(scene.mesh.texture.shape[:2])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    PM = (P["means"], P["scales"], P["quats"], P["opacity"], P["sh"])
    names = ["rasterize_mesh", "project", "bin_sort", "blend_forward", "zero_grads",
             "texture_backward", "blend_backward", "project_backward"]

    def step(ev=None):
        def mark(j):
            if ev is not None:
                ev[j].record(stream)
        mark(0)
        r.status_word.zero_()
        r.rasterize_mesh(mesh)
        mark(1)
        r.project(*PM)
        mark(2)
        r.bin_sort()
        mark(3)
        r.blend()
        mark(4)
        for v in grads.values():            # the caller zero-initialises gradients
            v.zero_()
        mark(5)
        # the backward pass as its three kernels, each bracketed by events
        for j, stg in ((6, lib.HM_BWD_TEXTURE), (7, lib.HM_BWD_BLEND), (8, lib.HM_BWD_PROJECT)):
            r.backward(*PM, dI, None, mesh=mesh, tex_grad=True, out=grads, stages=stg, zero=False)
            mark(j)

    for _ in range(max(3, args.warmup)):
        step()
        flush.fill_(1.0)
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(9)] for _ in range(args.steps)]
    _barrier(dist)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            step(events[k])
            flush.fill_(float(k))          # L2 flush between steps (outside the events)
        _barrier(dist)
    st, npairs, nitems = r.status()
    if st:
        raise RuntimeError(f"device status {st} during the timed region")

    # the same step captured once in a CUDA graph (the production path): the
    # headline number
    from paper_2506_06988_b300.render import GraphStep
    gs = GraphStep(r, PM, mesh, dL_drgb=dI, grads=grads, tex_grad=True)
    for _ in range(max(3, args.warmup)):
        gs.replay()
        flush.fill_(1.0)
    with ClockSampler(local) as gclk:
        graph_ms = _time_replays(gs, args.steps, flush, stream, dist)
    st, npairs, nitems = r.status()
    if st:
        raise RuntimeError(f"device status {st} during the timed graph replays")
    del gs
    gsf = GraphStep(r, PM, mesh)                      # forward only
    for _ in range(3):
        gsf.replay()
        flush.fill_(1.0)
    graph_fwd_ms = _time_replays(gsf, args.steps, flush, stream, dist)
    del gsf
    stage = np.array([[events[k][j].elapsed_time(events[k][j + 1]) for j in range(8)]
                      for k in range(args.steps)])           # ms
    step_ms_local = float(stage.sum(1).mean())
    step_ms = _max_over_ranks(step_ms_local, dist)
    fwd_ms = _max_over_ranks(float(stage[:, :4].sum(1).mean()), dist)
    stage_ms = {n: float(stage[:, j].mean()) for j, n in enumerate(names)}

    # algorithmic work of the blend (instrumented re-run, outside the timing)
    n_blended = int(r.n_contrib.to(torch.int64).sum().item())
    n_mesh_px = int(torch.isfinite(r.mesh_depth).sum().item())
    n_eval, n_exam = r.count_evaluations()
    peaks, peak_kind = _peaks()
    clocks = clk.summary()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s at the max clock
    frames = V * world
    value = frames * 1e3 / graph_ms
    mpx = value * 1920 * 1080 / 1e6
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    tsuf = f"<{tile[0]},{tile[1]}>"
    N, M = g.n, V * g.n
    K = (g.sh_degree + 1) ** 2
    # per single-kernel stage: (kernel, bound, algorithmic units, work per unit)
    kern = {
        "blend_forward": ("blend_fwd_kernel" + tsuf, "alu", n_eval, METHOD_FLOPS["blend_forward"],
                          "evaluated (pixel, Gaussian) pairs (inside 3 sigma), nominal count of the method"),
        "blend_backward": ("blend_bwd_kernel" + tsuf[:-1] + (",2>" if tuple(tile) == (16, 16) else ",1>"), "alu",
                           n_eval, METHOD_FLOPS["blend_backward"],
                           "evaluated (pixel, Gaussian) pairs (inside 3 sigma), nominal count of the method"),
        "project": ("project_kernel<3,false>", "hbm", N, 12 + 12 + 16 + 4 + 12 * K + V * 48, "Gaussians (params read + V records written, bytes)"),
        "project_backward": ("project_bwd_kernel<3,false>", "hbm", N, 2 * (12 + 12 + 16 + 4 + 12 * K) + 12 + 12 + 16 + 4 + 12 * K + V * 36,
                             "Gaussians (params read, grads read+written, V partial rows read, bytes)"),
        "texture_backward": ("texture_bwd_kernel", "hbm", n_mesh_px, 4 + 4 + 8 + 12, "mesh pixels (depth, T, uv, dL/dI read, bytes)"),
    }
    per_kernel = {}
    issue_peak = nsm * 4 * sm_max * 1e6 / 1e9          # warp instructions / s (G), one per SMSP per clock
    for st_name, (kname, bound, units, per, what) in kern.items():
        t = stage_ms[st_name] * 1e-3
        if bound == "alu":
            ach = units * per / t / 1e12
            src_units = n_eval if st_name == "blend_forward" else n_blended
            src = src_units * SOURCE_FLOPS[st_name] / t / 1e12
            per_kernel[st_name] = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": fp32_peak,
                                   "unit": "TFLOP/s", "frac": ach / fp32_peak, "units": units,
                                   "per_unit": per, "unit_kind": what, "ms": stage_ms[st_name],
                                   "source_count": {"per_unit": SOURCE_FLOPS[st_name], "units": src_units,
                                                    "unit_kind": ("evaluated pairs" if st_name == "blend_forward"
                                                                  else "blended pairs"),
                                                    "achieved": src, "frac": src / fp32_peak}}
            wi, dram = _captured(st_name, tile, {"evaluated_pairs": n_eval, "blended_pairs": n_blended},
                                 r.npix)
            per_kernel[st_name]["traffic"] = dram
            per_kernel[st_name]["issue"] = (
                {"warp_inst_per_launch": wi, "achieved_ginst_s": wi / t / 1e9, "peak_ginst_s": issue_peak,
                 "frac": wi / t / 1e9 / issue_peak,
                 "thread_inst_per_blended_pair": wi * 32 / max(n_blended, 1)}
                if wi is not None else None)
        else:
            ach = units * per / t / 1e9
            per_kernel[st_name] = {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": hbm,
                                   "unit": "GB/s", "frac": ach / hbm, "units": units, "per_unit": per,
                                   "unit_kind": what, "ms": stage_ms[st_name]}
    for st_name, e in per_kernel.items():
        # DRAM bytes read + written per launch from the committed ncu capture
        # (None when that kernel's sources differ from the captured ones)
        e.setdefault("traffic", None)
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    roof = dict(per_kernel[dom])
    roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on 3 of the 8 "
                              "views, scaled by pixels (profiles/blend_*_kernel_room1080p_3views.md)")
    roof["time_source"] = ("CUDA events around the kernel's library call in the eager step (the backward's "
                           "includes the zeroing of its per-record partial sums)")
    roof["peak_source"] = (f"FP32: {nsm} SMs x 128 lanes x 2 FLOP x {sm_max:.0f} MHz (unit counts x max clock)"
                           if roof["bound"] == "alu" else f"HBM copy bandwidth, {peak_kind}")
    if roof["bound"] == "alu" and clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = roof["achieved"] / (nsm * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    # count and emit each read every record (48 B); per pair the 8-B key
    # written and read back and the 4-B index written; per tile the counts,
    # offsets and ranges
    sort_bytes = M * 48 * 2 + npairs * (8 + 8 + 4) + r.ntiles * 16
    stage_roof = {"bin_sort": {"bytes": sort_bytes, "GB/s": sort_bytes / (stage_ms["bin_sort"] * 1e-3) / 1e9}}
    stage_roof["bin_sort"]["frac_of_hbm"] = stage_roof["bin_sort"]["GB/s"] / hbm
    # the mesh pass: per pixel the 28-B G-buffer (tri_id, depth, colour, UV)
    # written and up to 12 B of texels read
    mesh_bytes = V * 1920 * 1080 * (28 + 12)
    stage_roof["rasterize_mesh"] = {"bytes": mesh_bytes,
                                    "GB/s": mesh_bytes / (stage_ms["rasterize_mesh"] * 1e-3) / 1e9}
    stage_roof["rasterize_mesh"]["frac_of_hbm"] = stage_roof["rasterize_mesh"]["GB/s"] / hbm
    # frame roofline: each stage's floor (its algorithmic work at the peak of
    # the unit that bounds it) summed, against the measured graph step
    floors = {k: v["ms"] * v["frac"] for k, v in per_kernel.items()}
    floors.update({k: v["bytes"] / (hbm * 1e9) * 1e3 for k, v in stage_roof.items()})
    frame_roof = {"stage_floor_ms": floors, "floor_sum_ms": float(sum(floors.values())), "measured_ms": graph_ms,
                  "frac": float(sum(floors.values())) / graph_ms,
                  "note": "blend stages at the FP32 peak (they are bound by the half-rate ALU pipe: "
                          "compares, selects), the others at the measured HBM copy bandwidth"}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, scene, r, mesh, dev, dist, V * world)

    extra = {}
    if not args.no_extra:
        extra["batched16"] = run_batched16(args, dev, dist)
        extra["mip"] = run_mip(args, dev, dist)
        extra["prune"] = run_prune(args, dev, dist)
        extra["texture_opt"] = run_texture_opt(args, dev, dist)
        extra["plain"] = run_plain(args, dev, dist)
        extra["joint_opt"] = run_joint_opt(args, dev, dist)
        extra["large"] = run_large(args, dev, dist)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": graph_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "mpixel_per_s": mpx,
        "fwd": {"frames_per_s": frames * 1e3 / graph_fwd_ms, "ms_per_step": graph_fwd_ms,
                "mpixel_per_s": frames * 1e3 / graph_fwd_ms * 1920 * 1080 / 1e6,
                "eager_ms_per_step": fwd_ms},
        "launch": "one CUDA graph per step (GraphStep); stage_ms from the same step launched eagerly "
                  "with events between the stages",
        "eager": {"frames_per_s": frames * 1e3 / step_ms, "ms_per_step": step_ms},
        "stage_ms": stage_ms,
        "config": {"workload": WORKLOAD, "views": V, "width": 1920, "height": 1080, "gaussians": g.n,
                   "seed": int(scene.seed), "view_block": rank,
                   "sh_degree": g.sh_degree, "faces": len(scene.mesh.faces), "tile": list(tile),
                   "batch": r.opt.batch, "pairs": npairs, "mesh_items": nitems,
                   "device_mem_gb": torch.cuda.max_memory_allocated(dev) / 1e9,
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "parallelism": f"views per rank, {world} rank(s)"},
        "roofline": roof, "kernels": per_kernel, "stage_roofline_hbm": stage_roof, "frame_roofline": frame_roof,
        "blend_units": {"evaluated_pairs": n_eval, "examined_pairs": n_exam, "blended_pairs": n_blended},
        "peak_kind": peak_kind,
        "paper_context": {"hardware": "one V100", "hybrid_fps_mean": {"Deep Blending": 498, "ScanNet++": 231},
                          "what": "forward only, the CUDA rasteriser routine, trained models of real "
                                  "captures at an unstated resolution (Tab. 1); not this workload"},
        "clocks": gclk.summary(),
        "clocks_eager": clocks,
        "gpu_launches": sum(KERNELS_PER_STEP.values()) * args.steps,
    }
    if e2e is not None:
        line["e2e"] = e2e
    line.update(extra)
    if not args.no_cpu_baseline and rank == 0:
        from oracle import oracle as O
        t0 = time.perf_counter()
        fwd_s, fb_s, info = cpu_oracle_sample(scene, rows=128, crop=44, t_fixed=fixed_grad_cost(scene))
        line["cpu_baseline"] = {"value": 1.0 / fb_s, "unit": UNIT, "cores": O.num_threads(),
                                "kind": "oracle", "forward_frames_per_s": 1.0 / fwd_s,
                                "sample": f"one 1080p view: oracle forward over {info['rows']} rows "
                                          f"(+ full projection) and FP64 autograd backward over a "
                                          f"{info['crop']}x{info['crop']} block, scaled to a full frame "
                                          f"({time.perf_counter() - t0:.1f} s of CPU work)",
                                "config0_full": cpu_oracle_small()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _time_replays(gs, steps, flush, stream, dist):
    """Mean ms per replay of a GraphStep over `steps` replays, each bracketed
    by CUDA events on the launching stream, with an L2 flush (256 MB write)
    between replays outside the events; max over ranks."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    _barrier(dist)
    for k in range(steps):
        ev[k][0].record(stream)
        gs.replay()
        ev[k][1].record(stream)
        flush.fill_(float(k))
    _barrier(dist)
    return _max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dist)


STAGES = ["rasterize_mesh", "project", "bin_sort", "blend_forward", "zero_grads",
          "texture_backward", "blend_backward", "project_backward"]


def _eager_stage_ms(r, PM, mesh, dI, grads, flush, stream, steps):
    """Mean ms of each stage of a forward+backward frame launched stage by
    stage with CUDA events between the stages (L2 flushed between frames)."""
    import torch
    from paper_2506_06988_b300 import lib

    def step(ev=None):
        def mark(j):
            if ev is not None:
                ev[j].record(stream)
        mark(0)
        r.status_word.zero_()
        if r.has_mesh:
            r.rasterize_mesh(mesh)
        mark(1)
        r.project(*PM)
        mark(2)
        r.bin_sort()
        mark(3)
        r.blend()
        mark(4)
        for v in grads.values():
            v.zero_()
        mark(5)
        for j, stg in ((6, lib.HM_BWD_TEXTURE), (7, lib.HM_BWD_BLEND), (8, lib.HM_BWD_PROJECT)):
            r.backward(*PM, dI, None, mesh=mesh, tex_grad=True, out=grads, stages=stg, zero=False)
            mark(j)

    for _ in range(2):
        step()
        flush.fill_(1.0)
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(9)] for _ in range(steps)]
    for k in range(steps):
        step(events[k])
        flush.fill_(float(k))
    torch.cuda.synchronize()
    t = np.array([[events[k][j].elapsed_time(events[k][j + 1]) for j in range(8)] for k in range(steps)])
    return {n: float(t[:, j].mean()) for j, n in enumerate(STAGES)}


def run_batched16(args, dev, dist):
    """16 cameras of uneven resolution (4 each at 640x480, 1024x768, 1296x968,
    1920x1080) of a room with 1M Gaussians (SH degree 3 stored as FP16,
    widened in the kernels), 200k triangles (10% pruned) and a 4096^2 RGB8
    atlas, forward+backward (texel gradients included) as one CUDA graph;
    tile shape and staging batch picked by the autotuner on this scene."""
    import torch
    from paper_2506_06988_b300 import autotune, scenes
    from paper_2506_06988_b300.render import GraphStep, MeshInput
    scene = scenes.config3_scene()
    g = scene.gaussians
    P = tuple(torch.as_tensor(getattr(g, k), device=dev).contiguous()
              for k in ("means", "scales", "quats", "opacity", "sh"))
    mesh = MeshInput.from_numpy(scene.mesh, device=dev)
    npix = sum(c.width * c.height for c in scene.cameras)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4321)
    dI = torch.randn(3 * npix, device=dev, generator=gen) * 1e-3
    kw = dict(sh_f16=True, n_verts=len(scene.mesh.verts), n_faces=len(scene.mesh.faces),
              tex_shape=scene.mesh.texture.shape, bg=tuple(scene.bg), device=dev)
    t0 = time.perf_counter()
    res = autotune.tune(scene.cameras, g.n, g.sh_degree, P, mesh, dL_drgb=dI, tex_grad=True, **kw)
    tune_s = time.perf_counter() - t0
    r = res.renderer
    gs = GraphStep(r, P, mesh, dL_drgb=dI, tex_grad=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        gs.replay()
        flush.fill_(1.0)
    steps = max(5, min(args.steps, 30))
    ms = _time_replays(gs, steps, flush, stream, dist)
    st, npairs, _ = r.status()
    if st:
        raise RuntimeError(f"device status {st} in the batched replays")
    # both launch modes of the blend kernels at the tuned tile and batch: the
    # graph replay and the stage breakdown of an eager frame
    launches = {}
    grads = r.grad_buffers(scene.mesh.texture.shape[:2])
    for pers in (False, True):
        r.opt.persistent = int(pers)
        gsl = GraphStep(r, P, mesh, dL_drgb=dI, tex_grad=True)
        for _ in range(3):
            gsl.replay()
            flush.fill_(1.0)
        launches["persistent" if pers else "grid"] = {
            "ms_per_step": _time_replays(gsl, steps, flush, stream, dist),
            "stage_ms": _eager_stage_ms(r, P, mesh, dI, grads, flush, stream, max(3, steps // 3))}
        del gsl
    r.opt.persistent = int(res.persistent)
    V = len(scene.cameras)
    out = {"workload": "16 views of uneven resolution (4 x 640x480, 4 x 1024x768, 4 x 1296x968, "
                       "4 x 1920x1080), room with 1M Gaussians SH3 stored FP16, 200k triangles (10% pruned), "
                       "4096^2 RGB8 atlas; forward+backward with texel gradients, one CUDA graph per step",
           "frames_per_s": V * 1e3 / ms, "mpixel_per_s": npix * 1e3 / ms / 1e6, "ms_per_step": ms,
           "views": V, "pixels": npix, "gaussians": g.n, "faces": len(scene.mesh.faces), "pairs": npairs,
           "tile": list(res.tile), "batch": res.batch, "persistent": res.persistent, "steps": steps,
           "launches": launches,
           "autotune": {"seconds": tune_s,
                        "ms_per_frame": [[list(t), b, "persistent" if p else "grid", m] for t, b, p, m in res.table]}}
    del gs, r, res
    torch.cuda.empty_cache()
    return out


def run_mip(args, dev, dist):
    """The headline workload (8 x 1920x1080 room, 300k Gaussians SH3, 50k
    faces) with the Mip-Splatting back-end the paper also pairs with the
    mesh (Tab. 1): the 3D smoothing filter (variance from the 8 cameras'
    sampling rates, computed once like a training-time constant) and the 2D
    Mip filter with opacity compensation; forward+backward as one CUDA
    graph per step.  The 3D-filter kernel is timed on its own."""
    import torch
    from paper_2506_06988_b300 import scenes
    from paper_2506_06988_b300.render import GraphStep, MeshInput, Renderer
    scene = scenes.config1_scene()
    g = scene.gaussians
    P = tuple(torch.as_tensor(getattr(g, k), device=dev).contiguous()
              for k in ("means", "scales", "quats", "opacity", "sh"))
    mesh = MeshInput.from_numpy(scene.mesh, device=dev)
    r = Renderer(scene.cameras, g.n, g.sh_degree, n_verts=len(scene.mesh.verts),
                 n_faces=len(scene.mesh.faces), tex_shape=scene.mesh.texture.shape, bg=tuple(scene.bg),
                 mip=True, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        r.mip_filter_3d(P[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        r.mip_filter_3d(P[0])
    e1.record(stream)
    torch.cuda.synchronize()
    f3_ms = e0.elapsed_time(e1) / 20
    seen = float((r.filter_3d > 0).float().mean())
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    dI = torch.randn(3 * r.npix, device=dev, generator=gen) * 1e-3
    gs = GraphStep(r, P, mesh, dL_drgb=dI, tex_grad=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        gs.replay()
        flush.fill_(1.0)
    steps = max(5, min(args.steps, 30))
    ms = _time_replays(gs, steps, flush, stream, dist)
    st, npairs, _ = r.status()
    if st:
        raise RuntimeError(f"device status {st} in the Mip replays")
    gf = GraphStep(r, P, mesh)
    for _ in range(3):
        gf.replay()
        flush.fill_(1.0)
    ms_f = _time_replays(gf, steps, flush, stream, dist)
    V = len(scene.cameras)
    out = {"workload": "Mip-Splatting back-end on the headline room (8 x 1920x1080, 300k Gaussians SH3, "
                       "50k faces): 3D smoothing filter (s2 = 0.2, from the 8 cameras) + 2D Mip filter "
                       "(kernel 0.1, opacity compensation); forward+backward, one CUDA graph per step",
           "frames_per_s": V * 1e3 / ms, "ms_per_step": ms, "fwd_frames_per_s": V * 1e3 / ms_f,
           "fwd_ms_per_step": ms_f, "pairs": npairs, "filter_3d_ms": f3_ms,
           "filter_3d_seen_fraction": seen, "steps": steps}
    del gs, gf, r
    torch.cuda.empty_cache()
    return out


def run_prune(args, dev, dist):
    """The mesh-pruning metrics (Sec. 3.3, Algorithm 1 stage 1) by
    hm_mesh_prune with the paper's parameters (alpha_normal 20, alpha_area
    50, 45 degrees, alpha_group 100):
    * ``room``: the headline room's 50k-face mesh (coincident vertices welded
      so walls share their corner edges) seen by its 8 cameras at 1920x1080,
      pixel -> triangle maps from hm_rasterize_mesh, seeded prior normal maps;
    * ``large``: the 2x2-room mesh of 1M triangles (15% pruned), geometric
      metrics only (angle, area, pieces).
    The call synchronises (the piece labelling iterates on the host)."""
    import torch
    from paper_2506_06988_b300 import lib, scenes
    from paper_2506_06988_b300.render import MeshInput, Renderer
    out = {"workload": "mesh-pruning metrics (normal-map variation, adjacent angle, area rank, "
                       "small pieces) with the paper's parameters"}
    p = lib.prune_params()

    def weld(m):
        uniq, inv = np.unique(np.asarray(m.verts, np.float32), axis=0, return_inverse=True)
        return uniq, inv.reshape(-1)[np.asarray(m.faces)].astype(np.int32)

    def time_prune(cams, verts, faces, tri, nrm, reps):
        v = torch.as_tensor(verts, device=dev).contiguous()
        f = torch.as_tensor(faces, device=dev).contiguous()
        cam_arr = lib.cameras(cams) if cams else None
        ws = torch.empty(max(1, lib.hm_mesh_prune_workspace_size(cam_arr, len(verts), len(faces))),
                         dtype=torch.uint8, device=dev)
        flags = torch.empty(len(faces), dtype=torch.uint8, device=dev)
        label = torch.empty(len(faces), dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        call = lambda: lib.check(lib.hm_mesh_prune(cam_arr, v, len(verts), f, len(faces), tri, nrm, p, flags,  # noqa: E731
                                                   label, ws, ws.numel(), stream), "hm_mesh_prune")
        call()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            call()
            ts.append((time.perf_counter() - t0) * 1e3)
        fl = flags.cpu().numpy()
        return float(np.median(ts)), {name: int(((fl & b) > 0).sum()) for name, b in
                                      (("normal", 1), ("angle", 2), ("area", 4), ("group", 8))}, int((fl == 0).sum())

    scene = scenes.config1_scene()
    verts, faces = weld(scene.mesh)
    mesh = MeshInput.from_numpy(scene.mesh, device=dev)
    g = scene.gaussians
    r = Renderer(scene.cameras, g.n, g.sh_degree, n_verts=len(scene.mesh.verts), n_faces=len(scene.mesh.faces),
                 tex_shape=scene.mesh.texture.shape, bg=tuple(scene.bg), device=dev)
    r.rasterize_mesh(mesh)
    nm = torch.as_tensor(np.concatenate([n.reshape(-1) for n in scenes.prior_normal_maps(scene.cameras, seed=9)]),
                         device=dev)
    ms, counts, kept = time_prune(scene.cameras, verts, faces, r.tri_id, nm, 5)
    npix = sum(c.width * c.height for c in scene.cameras)
    out["room"] = {"faces": len(faces), "views": len(scene.cameras), "pixels": npix, "ms": ms,
                   "mpixel_per_s": npix / ms / 1e3, "removed": counts, "kept": kept}
    del r, nm, mesh
    big = scenes.room_scene(4, rooms=(2, 2), n_tris=1_000_000, prune_frac=0.15, atlas=64, n_gauss=1,
                            resolutions=((64, 64),))
    verts, faces = weld(big.mesh)
    ms, counts, kept = time_prune(None, verts, faces, None, None, 5)
    out["large"] = {"faces": len(faces), "ms": ms, "mfaces_per_s": len(faces) / ms / 1e3, "removed": counts,
                    "kept": kept}
    torch.cuda.empty_cache()
    return out


def run_texture_opt(args, dev, dist):
    """Texture optimisation from images alone (the texture initialisation of
    Sec. 3.3): the headline room's mesh (50k faces) and 2048^2 atlas as FP32
    texels, 8 cameras at 1920x1080; targets rendered from the true texture,
    optimisation from a grey texture: per step the mesh-only render, the
    Eq. 3 loss, the texel gradient and Adam, all in library kernels."""
    import torch
    from paper_2506_06988_b300 import scenes
    from paper_2506_06988_b300.render import MeshInput
    from paper_2506_06988_b300.texture_opt import TextureOptimizer
    scene = scenes.config1_scene()
    mesh = MeshInput.from_numpy(scene.mesh, device=dev)
    true = TextureOptimizer(scene.cameras, mesh, torch.zeros(3 * sum(c.width * c.height for c in scene.cameras),
                                                             device=dev), bg=tuple(scene.bg), device=dev)
    target = true.render().clone()
    grey = MeshInput(mesh.verts, mesh.uvs, mesh.faces, torch.full(tuple(scene.mesh.texture.shape), 0.5,
                                                                  dtype=torch.float32, device=dev))
    opt = TextureOptimizer(scene.cameras, grey, target, lr=0.02, bg=tuple(scene.bg), device=dev)
    del true
    first = float(opt.step(check=True)[3])
    for _ in range(2):
        opt.step()
    steps = max(5, min(args.steps, 20))
    stream = torch.cuda.current_stream()

    def timed(n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        _barrier(dist)
        for k in range(n):
            ev[k][0].record(stream)
            t_ = opt.step()
            ev[k][1].record(stream)
        _barrier(dist)
        return _max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dist), t_
    ms_eager, _ = timed(steps)
    opt.capture()
    for _ in range(2):
        opt.step()
    ms, terms = timed(steps)
    last = float(opt.step(check=True)[3])
    V = len(scene.cameras)
    out = {"workload": "texture-only optimisation: room mesh (50k faces), 2048^2 FP32 texels, 8 x 1920x1080, "
                       "Eq. 3 loss, Adam; one CUDA graph per step",
           "steps_per_s": 1e3 / ms, "ms_per_step": ms, "frames_per_s": V * 1e3 / ms,
           "eager_ms_per_step": ms_eager,
           "loss_first": first, "loss_last": last, "steps": opt.t}
    del opt
    torch.cuda.empty_cache()
    return out


def run_joint_opt(args, dev, dist):
    """One joint optimisation step of Gaussians and FP32 texels (Sec. 3.4):
    the room at 1296x968 with 500k Gaussians (SH degree 3) and a 2048^2 FP32
    learnable texture, against a target rendered from perturbed parameters
    (means + N(0, 0.01), colours + N(0, 0.05)); activations in PyTorch; Adam
    (PyTorch's fused kernel).  Two losses:
    * ``l1``: a plain L1 in PyTorch through the HybridRender autograd Function;
    * ``paper``: the joint loss of Eq. 3 + Sec. 3.4 (0.8 L1 + 0.2 D-SSIM +
      0.1 transmittance-aware texture loss) by the fused hm_hybrid_loss, its
      dL/dI_h and dL/dI_m fed straight to hm_blend_backward."""
    import torch
    from paper_2506_06988_b300 import lib, scenes
    from paper_2506_06988_b300.render import HybridRender, MeshInput, Renderer
    from paper_2506_06988_b300.schedule import texture_loss_weight
    scene = scenes.config2_scene()
    g = scene.gaussians
    tgt = scenes.config2_target_params(scene)
    mesh = MeshInput.from_numpy(scene.mesh, device=dev)
    r = Renderer(scene.cameras, g.n, g.sh_degree, n_verts=len(scene.mesh.verts),
                 n_faces=len(scene.mesh.faces), tex_shape=scene.mesh.texture.shape,
                 bg=tuple(scene.bg), device=dev)
    T = lambda a: torch.as_tensor(a, device=dev).contiguous()  # noqa: E731
    r.render(T(tgt.means), T(tgt.scales), T(tgt.quats), T(tgt.opacity), T(tgt.sh), mesh)
    target = r.rgb.clone()
    means = T(g.means).requires_grad_()
    log_s = torch.log(T(g.scales)).requires_grad_()
    quats = T(g.quats).requires_grad_()
    logit = torch.logit(T(g.opacity)).requires_grad_()
    sh = T(g.sh).requires_grad_()
    tex = mesh.texture.clone().requires_grad_()
    params = [means, log_s, quats, logit, sh, tex]
    init = [p.detach().clone() for p in params]
    opt = torch.optim.Adam(params, lr=1e-4, fused=True)
    lp = lib.loss_params(lambda_t=texture_loss_weight(5000))
    mesh_t = MeshInput(mesh.verts, mesh.uvs, mesh.faces, tex.detach())

    def step_l1():
        opt.zero_grad(set_to_none=False)
        rgb, _ = HybridRender.apply(r, mesh, means, torch.exp(log_s), quats, torch.sigmoid(logit), sh, tex)
        loss = (rgb - target).abs().mean()
        loss.backward()
        opt.step()
        return loss

    def step_paper():
        opt.zero_grad(set_to_none=False)
        s_, o_ = torch.exp(log_s), torch.sigmoid(logit)
        P = (means.detach(), s_.detach(), quats.detach(), o_.detach(), sh.detach())
        r.render(*P, mesh_t)
        terms, dI, dM = r.loss(target, lp)
        gr = r.backward(*P, dI, None, mesh=mesh_t, tex_grad=True, dL_dmesh=dM)
        torch.autograd.backward([s_, o_], [gr["scales"], gr["opacity"]])
        means.grad.add_(gr["means"])
        quats.grad.add_(gr["quats"])
        sh.grad.add_(gr["sh"])
        tex.grad.add_(gr["texture"])
        opt.step()
        return terms[3]

    stream = torch.cuda.current_stream()
    out = {"workload": "joint optimisation step: room at 1296x968, 500k Gaussians SH3, 2048^2 FP32 "
                       "learnable texels vs a target rendered from perturbed parameters; fused Adam"}
    W, H = scene.cameras[0].width, scene.cameras[0].height
    for name, step in (("l1", step_l1), ("paper", step_paper)):
        with torch.no_grad():
            for p, p0 in zip(params, init):
                p.copy_(p0)
        opt = torch.optim.Adam(params, lr=1e-4, fused=True)
        first = float(step().item())
        for _ in range(2):
            step()
        steps = max(5, min(args.steps, 20))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        _barrier(dist)
        for k in range(steps):
            ev[k][0].record(stream)
            loss = step()
            ev[k][1].record(stream)
        _barrier(dist)
        ms = _max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dist)
        out[name] = {"frames_per_s": 1e3 / ms, "ms_per_step": ms, "mpixel_per_s": W * H * 1e3 / ms / 1e6,
                     "loss_first": first, "loss_last": float(loss.item()), "steps": steps}
    # the same paper-loss step as one CUDA graph (JointTrainStep: activations,
    # render, fused loss, gradients and Adam all in library kernels)
    from paper_2506_06988_b300.train import JointTrainStep
    with torch.no_grad():
        for p, p0 in zip(params, init):
            p.copy_(p0)
    pj = dict(means=means.detach().clone(), log_scales=log_s.detach().clone(), quats=quats.detach().clone(),
              logit=logit.detach().clone(), sh=sh.detach().clone())
    mesh_j = MeshInput(mesh.verts, mesh.uvs, mesh.faces, tex.detach().clone())
    ts = JointTrainStep(r, pj, mesh_j, target, lrs=dict(means=1e-4, log_scales=1e-4, quats=1e-4, logit=1e-4,
                                                        sh=1e-4, texture=1e-4),
                        eps=1e-8, lambda_t=texture_loss_weight(5000))
    first = float(ts.step()[3])
    for _ in range(2):
        ts.step()
    steps = max(5, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    _barrier(dist)
    for k in range(steps):
        ev[k][0].record(stream)
        terms = ts.step()
        ev[k][1].record(stream)
    _barrier(dist)
    ms = _max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dist)
    out["paper_graph"] = {"frames_per_s": 1e3 / ms, "ms_per_step": ms, "mpixel_per_s": W * H * 1e3 / ms / 1e6,
                          "loss_first": first, "loss_last": float(terms[3]), "steps": steps,
                          "loss": "as 'paper', the whole step (activations, render, loss, gradients, Adam) "
                                  "one CUDA graph replay (JointTrainStep)"}
    del ts
    out["l1"]["loss"] = "mean |I_h - I| in PyTorch, HybridRender autograd"
    out["paper"]["loss"] = ("0.8 L1 + 0.2 (1 - SSIM 11x11) + 0.1 M_T |I - I_m|^2 by the fused "
                            "hm_hybrid_loss (lambda_t of iteration 5000 of the warm-up schedule)")
    # the fused loss alone (forward terms and both gradients, one frame):
    # n_l calls captured in one CUDA graph, so the device time is measured
    # rather than the host's call rate
    for _ in range(3):
        r.loss(target, lp)
    torch.cuda.synchronize()
    n_l = 20
    lg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(lg):
        for _ in range(n_l):
            r.loss(target, lp)
    lg.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lg.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    lm = e0.elapsed_time(e1) / n_l
    # algorithmic bytes: read I_h, I, I_m (3 planes each) + T + depth, write
    # dL/dI_h and dL/dI_m; the SSIM statistics (9 floats per pixel) are
    # written once and read once by the gradient pass
    npx = W * H
    alg = npx * 4 * (3 + 3 + 3 + 1 + 1 + 3 + 3 + 2 * 9)
    out["loss_kernel"] = {"ms": lm, "alg_bytes": alg, "achieved_gbs": alg / lm / 1e6,
                          "launches": 4, "note": "ssim_fwd + ssim_bwd + two reduction levels over 32x32 tiles "
                                                 "x 3 channels, 20 calls in one CUDA graph (inputs L2-resident)"}
    del r, opt
    torch.cuda.empty_cache()
    out["loss_kernel_8x1080p"] = time_loss_8x1080p(dev)
    return out


def time_loss_8x1080p(dev):
    """hm_hybrid_loss on 8 views of 1920x1080 (each input plane 199 MB, past
    the L2): the Eq. 3 loss with D-SSIM, and the L1-only pointwise path."""
    import torch
    from paper_2506_06988_b300 import lib, scenes
    cams = lib.cameras([scenes._identity_cam(1920, 1080) for _ in range(8)])
    npx = 8 * 1920 * 1080
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    x = torch.rand(3 * npx, device=dev, generator=gen)
    y = torch.rand(3 * npx, device=dev, generator=gen)
    ws = torch.empty(lib.hm_hybrid_loss_workspace_size(cams), dtype=torch.uint8, device=dev)
    lout = torch.empty(4, dtype=torch.float64, device=dev)
    dI = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    res = {}
    for name, lam, alg_per_px in (("ssim", 0.2, 4 * (3 + 3 + 3 + 2 * 9)), ("l1_only", 0.0, 4 * (3 + 3 + 3))):
        lp = lib.loss_params(lambda_ssim=lam, lambda_t=0.0)

        def call():
            lib.check(lib.hm_hybrid_loss(cams, x, y, None, None, None, lp, lout, dI, None, ws, ws.numel(),
                                         stream.cuda_stream), "hm_hybrid_loss")
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        alg = npx * alg_per_px
        res[name] = {"ms": ms, "alg_bytes": alg, "achieved_gbs": alg / ms / 1e6}
    res["note"] = ("algorithmic bytes: I_h, I read, dL/dI_h written; with D-SSIM also the 9 window "
                   "statistics per pixel written and read once; back-to-back calls, inputs past the L2")
    del x, y, ws, dI
    torch.cuda.empty_cache()
    return res


def run_large(args, dev, dist):
    """The large scene: 4 connected rooms (~1M faces, 15% pruned, 4096^2
    atlas), 3M Gaussians SH3, 8 views at 3840x2160, forward+backward with
    texel gradients through the chunked renderer (two views at a time; the
    backward pass recomputes each chunk's sorted lists instead of storing
    them)."""
    import torch
    from paper_2506_06988_b300 import scenes
    from paper_2506_06988_b300.render import ChunkedRenderer, MeshInput
    torch.cuda.reset_peak_memory_stats(dev)
    base_mem = torch.cuda.memory_allocated(dev)
    scene = scenes.config4_scene()
    g = scene.gaussians
    P = tuple(torch.as_tensor(getattr(g, k), device=dev).contiguous()
              for k in ("means", "scales", "quats", "opacity", "sh"))
    mesh = MeshInput.from_numpy(scene.mesh, device=dev)
    chunk = 2
    cr = ChunkedRenderer(scene.cameras, g.n, g.sh_degree, chunk=chunk, n_verts=len(scene.mesh.verts),
                         n_faces=len(scene.mesh.faces), tex_shape=scene.mesh.texture.shape,
                         bg=tuple(scene.bg), device=dev)
    cr.render(*P, mesh)
    gen = torch.Generator(device=dev)
    gen.manual_seed(777)
    dI = torch.randn(3 * cr.npix, device=dev, generator=gen) * 1e-3
    grads = cr.grad_buffers(scene.mesh.texture.shape[:2])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    steps = max(3, min(args.steps, 10))
    for mode in ("fwd", "fwd_bwd"):
        for _ in range(2):
            cr.forward(*P, mesh)
            if mode == "fwd_bwd":
                cr.backward(*P, dI, mesh=mesh, tex_grad=True, out=grads)
            flush.fill_(1.0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        _barrier(dist)
        for k in range(steps):
            ev[k][0].record(stream)
            cr.forward(*P, mesh)
            if mode == "fwd_bwd":
                cr.backward(*P, dI, mesh=mesh, tex_grad=True, out=grads)
            ev[k][1].record(stream)
            flush.fill_(float(k))
        _barrier(dist)
        res[mode] = _max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dist)
    if cr.status():
        raise RuntimeError("device status set in the large-scene run")
    npairs = [int(r.n_pairs.item()) for r in cr._renderers.values()]
    chunk_mem = (torch.cuda.max_memory_allocated(dev) - base_mem) / 1e9
    npix = cr.npix
    del cr, grads
    torch.cuda.empty_cache()
    # the same 8 views in one renderer and one CUDA graph per step: on a GPU
    # with this much memory every list of every view stays resident
    from paper_2506_06988_b300.render import GraphStep, Renderer
    torch.cuda.reset_peak_memory_stats(dev)
    base1 = torch.cuda.memory_allocated(dev)
    r1 = Renderer(scene.cameras, g.n, g.sh_degree, n_verts=len(scene.mesh.verts), n_faces=len(scene.mesh.faces),
                  tex_shape=scene.mesh.texture.shape, bg=tuple(scene.bg), device=dev)
    res1 = {}
    for mode in ("fwd", "fwd_bwd"):
        gs = GraphStep(r1, P, mesh, dL_drgb=dI if mode == "fwd_bwd" else None, tex_grad=True)
        for _ in range(2):
            gs.replay(check=True)
            flush.fill_(1.0)
        res1[mode] = _time_replays(gs, steps, flush, stream, dist)
        del gs
    st1, npairs1, _ = r1.status()
    if st1:
        raise RuntimeError("device status set in the unchunked large-scene run")
    nv = len(scene.cameras)
    unchunked = {"fwd": {"frames_per_s": nv * 1e3 / res1["fwd"], "ms_per_step": res1["fwd"]},
                 "fwd_bwd": {"frames_per_s": nv * 1e3 / res1["fwd_bwd"], "ms_per_step": res1["fwd_bwd"]},
                 "pairs": npairs1, "device_mem_gb": (torch.cuda.max_memory_allocated(dev) - base1) / 1e9,
                 "launch": "one renderer over the 8 views, one CUDA graph per step (GraphStep)"}
    del r1
    V = len(scene.cameras)
    out = {"workload": "4 connected rooms, 3M Gaussians SH3, ~1M faces (15% pruned), 4096^2 atlas, "
                       "8 x 3840x2160; chunked renderer (2 views per chunk, sorted lists recomputed in "
                       "the backward)",
           "fwd": {"frames_per_s": V * 1e3 / res["fwd"], "ms_per_step": res["fwd"],
                   "mpixel_per_s": npix * 1e3 / res["fwd"] / 1e6},
           "fwd_bwd": {"frames_per_s": V * 1e3 / res["fwd_bwd"], "ms_per_step": res["fwd_bwd"],
                       "mpixel_per_s": npix * 1e3 / res["fwd_bwd"] / 1e6},
           "gaussians": g.n, "faces": len(scene.mesh.faces), "views": V, "chunk": chunk,
           "pairs_last_chunk": npairs, "steps": steps, "device_mem_gb": chunk_mem,
           "unchunked": unchunked}
    del dI
    torch.cuda.empty_cache()
    return out


def run_plain(args, dev, dist):
    """The single-view, unbatched plain renderer: one 1920x1080 view of the
    Gaussian-only comparison room (1.2M Gaussians, the walls as flat
    Gaussians, no mesh), frames launched eagerly one at a time."""
    import torch
    from paper_2506_06988_b300 import scenes
    from paper_2506_06988_b300.render import Renderer
    scene = scenes.config1_plain_scene()
    g = scene.gaussians
    P = tuple(torch.as_tensor(getattr(g, k), device=dev).contiguous()
              for k in ("means", "scales", "quats", "opacity", "sh"))
    cams = scene.cameras[:1]
    r = Renderer(cams, g.n, g.sh_degree, bg=tuple(scene.bg), device=dev)
    r.render(*P)
    gen = torch.Generator(device=dev)
    gen.manual_seed(99)
    dI = torch.randn(3 * r.npix, device=dev, generator=gen) * 1e-3
    grads = r.grad_buffers()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    steps = max(5, min(args.steps, 30))
    res = {}
    for mode in ("fwd", "fwd_bwd"):
        for _ in range(3):
            r.forward(*P)
            if mode == "fwd_bwd":
                r.backward(*P, dI, out=grads)
            flush.fill_(1.0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        _barrier(dist)
        for k in range(steps):
            ev[k][0].record(stream)
            r.forward(*P)
            if mode == "fwd_bwd":
                r.backward(*P, dI, out=grads)
            ev[k][1].record(stream)
            flush.fill_(float(k))
        _barrier(dist)
        res[mode] = _max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), dist)
    st, npairs, _ = r.status()
    if st:
        raise RuntimeError(f"device status {st} in the plain renderer")
    out = {"workload": "plain renderer: one 1920x1080 view, Gaussian-only room (1.2M Gaussians SH3, "
                       "walls as flat Gaussians, no mesh), single view, unbatched, eager launches",
           "fwd": {"frames_per_s": 1e3 / res["fwd"], "ms_per_frame": res["fwd"],
                   "mpixel_per_s": 1920 * 1080 * 1e3 / res["fwd"] / 1e6},
           "fwd_bwd": {"frames_per_s": 1e3 / res["fwd_bwd"], "ms_per_frame": res["fwd_bwd"],
                       "mpixel_per_s": 1920 * 1080 * 1e3 / res["fwd_bwd"] / 1e6},
           "gaussians": g.n, "pairs": npairs, "steps": steps}
    del r, grads
    torch.cuda.empty_cache()
    return out


def run_e2e(args, scene, r, mesh, dev, dist, frames):
    """A training step through the public API (GraphStep with a target:
    forward, L1 loss by hm_hybrid_loss, backward with the texel gradients,
    all in one CUDA graph).  Every step copies its data -- the 8 target
    images, uint8 codes the loss kernels read directly -- from pinned host
    memory and reads its loss back (after the next step is queued, as an asynchronous
    training loop logs it); the Gaussian parameters and the mesh are the
    model's state and stay resident, as in a training loop.  The copy of
    step k+1 runs on a copy stream into a second target buffer (a second
    graph) while step k computes (double buffering, as a data loader's
    prefetch does); each step still moves its own images across the bus
    inside the timed region."""
    import torch
    from paper_2506_06988_b300 import lib
    from paper_2506_06988_b300.render import GraphStep
    g = scene.gaussians
    names = ("means", "scales", "quats", "opacity", "sh")
    params = [torch.as_tensor(getattr(g, k)).to(dev).contiguous() for k in names]
    tgt_host = (torch.rand(3 * r.npix, generator=torch.Generator().manual_seed(5)) * 255).to(torch.uint8).pin_memory()
    bufs = [tgt_host.to(dev) for _ in range(2)]
    loss_host = [torch.empty(4, dtype=torch.float64).pin_memory() for _ in range(2)]
    h2d = tgt_host.numel() * tgt_host.element_size()
    d2h = loss_host[0].numel() * loss_host[0].element_size()
    lp = lib.loss_params(lambda_ssim=0.0, lambda_t=0.0)
    grads = r.grad_buffers(tuple(mesh.texture.shape[:2]))
    # each graph also copies its loss terms to its pinned host buffer
    graphs = [GraphStep(r, params, mesh, target=b, loss_params=lp, grads=grads, tex_grad=True, loss_host=lh)
              for b, lh in zip(bufs, loss_host)]
    compute = torch.cuda.current_stream()
    copy = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    landed = [torch.cuda.Event(), torch.cuda.Event()]
    losses = []

    def issue_copy(k):
        with torch.cuda.stream(copy):
            copy.wait_event(used[k % 2])           # the step that last read this buffer is done
            bufs[k % 2].copy_(tgt_host, non_blocking=True)
            copied[k % 2].record(copy)

    def step(k):
        # step k is queued before step k - 1's loss is waited for, so the
        # device never idles on the host's read
        gs = graphs[k % 2]
        compute.wait_event(copied[k % 2])
        issue_copy(k + 1)                          # prefetch the next step's images
        gs.replay()
        used[k % 2].record(compute)
        landed[k % 2].record(compute)                 # the graph's last node wrote loss_host[k % 2]

    def read(k):
        landed[k % 2].synchronize()
        losses.append(float(loss_host[k % 2][3]))

    def run(k0, k1):
        for k in range(k0, k1):
            step(k)
            if k > k0:
                read(k - 1)
        read(k1 - 1)

    for ev in used:
        ev.record(compute)
    issue_copy(0)
    run(0, 3)
    st, _, _ = r.status()
    if st:
        raise RuntimeError(f"renderer status {st:#x} in the end-to-end step")
    n = max(10, min(args.steps, 50))
    _barrier(dist)
    t0 = time.perf_counter()
    run(3, 3 + n)
    _barrier(dist)
    sec = _max_over_ranks((time.perf_counter() - t0) / n, dist)
    torch.cuda.synchronize()
    return {"value": frames / sec, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": sec * 1e3,
            "losses_read": len(losses),
            "api": "GraphStep(target=uint8 images, L1 loss, loss_host=pinned buffer) replay, the graph's last "
                   "node copying the loss to pinned host memory, + every step's loss read back (step k's "
                   "read waited for after step k + 1 is queued); the step's images copied from pinned host "
                   "memory, double-buffered (next step's copy overlaps this step's compute); parameters "
                   "resident"}


def run_leg(args):
    import torch
    from paper_2506_06988_b300 import lib
    rank, world, local, dist = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lib.load()
    fn = {"batched16": run_batched16, "mip": run_mip, "prune": run_prune, "texture_opt": run_texture_opt,
          "plain": run_plain,
          "joint_opt": run_joint_opt,
          "large": run_large}
    out = fn[args.leg](args, dev, dist)
    if rank == 0:
        print(json.dumps({"leg": args.leg, **out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--views", type=int, default=8, help="fewer views: small case for profiling")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", default="16x16")
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--leg", default=None, choices=["batched16", "mip", "prune", "texture_opt", "plain", "joint_opt",
                                                          "large"],
                    help="run only this secondary workload and print its JSON (for profiling)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 16-view batched, plain single-view, joint-optimisation and "
                         "large-scene lines")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.leg:
        run_leg(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
