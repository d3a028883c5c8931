"""hm_blend_backward_noalloc: the backward pass for callers that cannot
allocate device memory (code inside a stream capture, a plug-in whose host
owns the allocator, a real-time loop), with its scratch in the library's
static device array.  Its gradients must equal those of hm_blend_backward
with a caller workspace, on two calls in a row (the array keeps the previous
call's contents, so the second call checks that the entry point clears what
it needs), with a mesh-colour gradient dL_dmesh passed through.  A context
reset moves the array; a call after the reset must find it again.  The file
sorts last so a run that stops at the first failure has run every other test
already; it also passes alone in a fresh process.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from paper_2506_06988_b300 import lib, scenes
from paper_2506_06988_b300.render import MeshInput, Renderer

pytestmark = pytest.mark.gpu


def _scene():
    s = scenes.config0_scene(seed=3)
    s.mesh.texture = s.mesh.texture.astype(np.float32) / 255.0
    s.bg = np.array([0.1, 0.2, 0.3], np.float32)
    return s


def _grads_noalloc(r, P, mesh, dI, dT, dM=None):
    th, tw = mesh.texture.shape[:2]
    g = r.grad_buffers((th, tw))
    r.opt.bwd_stages = 0
    st = lib.hm_blend_backward_noalloc(
        r.cams, r.n, P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], r.sh_degree,
        r.sh_format, r.records, r.pair_vals, r.ranges, r.mesh_depth, r.mesh_rgb, r.uv, tw, th,
        r.opt, r.T, r.last_idx, dI, dT, g["means"], g["scales"], g["quats"], g["opacity"], g["sh"],
        g["texture"], r.status_word, torch.cuda.current_stream().cuda_stream, dL_dmesh=dM)
    lib.check(st, "hm_blend_backward_noalloc")
    return g


def test_noalloc_backward_matches_workspace_backward_twice():
    s = _scene()
    g = s.gaussians
    dev = "cuda"
    P = {k: torch.as_tensor(getattr(g, k), device=dev).contiguous() for k in ("means", "scales", "quats", "opacity", "sh")}
    mesh = MeshInput.from_numpy(s.mesh, device=dev)
    r = Renderer(s.cameras, g.n, g.sh_degree, n_verts=len(s.mesh.verts), n_faces=len(s.mesh.faces),
                 tex_shape=s.mesh.texture.shape, bg=tuple(s.bg), device=dev)
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    dI = torch.randn(3 * r.npix, device=dev, generator=gen)
    dT = torch.randn(r.npix, device=dev, generator=gen)
    dM = torch.randn(3 * r.npix, device=dev, generator=gen)
    ref = r.backward(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], dI, dT, mesh=mesh,
                     tex_grad=True, overlap=False, dL_dmesh=dM)
    for _ in range(2):
        got = _grads_noalloc(r, P, mesh, dI, dT, dM)
        torch.cuda.synchronize()
        for k, v in ref.items():
            # same kernels; only the order of FP32 atomic additions may differ
            tol = 1e-5 * float(v.abs().max()) + 1e-12
            assert torch.allclose(got[k], v, rtol=1e-5, atol=tol), k


def test_noalloc_rejects_problems_above_its_static_scratch():
    cams = lib.cameras([scenes._identity_cam(16, 16)])
    o = lib.options()
    n_max = (lib.HM_BWD_NOALLOC_BYTES - 256) // (9 * 4)
    st = lib.hm_blend_backward_noalloc(cams, n_max + 1, 16, 16, 16, 16, 16, 0, lib.HM_SH_F32, 16, 16,
                                       16, None, None, None, 0, 0, o, 16, 16, 16, None, 16, 16, 16, 16,
                                       16, None, None, 0)
    assert st == lib.HM_ERR_INVALID_ARG
    assert "static array" in lib.last_error()


_RESET_CHILD = textwrap.dedent("""
    import ctypes, os, sys
    import numpy as np
    import torch
    sys.path.insert(0, os.environ["HM_ROOT"])
    from paper_2506_06988_b300 import lib
    from paper_2506_06988_b300.render import MeshInput, Renderer
    sys.path.insert(0, os.path.join(os.environ["HM_ROOT"], "tests"))
    import test_zz_no_alloc as T

    s = T._scene()
    g = s.gaussians
    P = {k: torch.as_tensor(getattr(g, k), device="cuda").contiguous()
         for k in ("means", "scales", "quats", "opacity", "sh")}
    mesh = MeshInput.from_numpy(s.mesh, device="cuda")
    r = Renderer(s.cameras, g.n, g.sh_degree, n_verts=len(s.mesh.verts), n_faces=len(s.mesh.faces),
                 tex_shape=s.mesh.texture.shape, bg=tuple(s.bg), device="cuda")
    r.render(P["means"], P["scales"], P["quats"], P["opacity"], P["sh"], mesh)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    dI = torch.randn(3 * r.npix, device="cuda", generator=gen)
    first = T._grads_noalloc(r, P, mesh, dI, None)
    torch.cuda.synchronize()
    want = {k: v.cpu().numpy() for k, v in first.items()}
    th, tw = mesh.texture.shape[:2]
    # every input of the call, as host bytes
    ins = dict(means=P["means"], scales=P["scales"], quats=P["quats"], opacity=P["opacity"],
               sh=P["sh"], records=r.records, pair_vals=r.pair_vals, ranges=r.ranges,
               mesh_depth=r.mesh_depth, mesh_rgb=r.mesh_rgb, uv=r.uv, T=r.T,
               last_idx=r.last_idx, dI=dI)
    host = {k: v.contiguous().cpu().numpy().tobytes() for k, v in ins.items()}
    outs = {k: v.numel() * v.element_size() for k, v in first.items()}
    torch.cuda.synchronize()

    # end this process's context: the library's module, and its static
    # array, are loaded again at the next call, possibly at another address
    rt = ctypes.CDLL("libcudart.so.13")
    assert rt.cudaDeviceReset() == 0
    def dev_alloc(nbytes):
        p = ctypes.c_void_p()
        assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(max(nbytes, 16))) == 0
        return p
    d = {}
    for k, b in host.items():
        d[k] = dev_alloc(len(b))
        assert rt.cudaMemcpy(d[k], ctypes.c_char_p(b), ctypes.c_size_t(len(b)), 1) == 0
    o = {k: dev_alloc(n) for k, n in outs.items()}
    for k, n in outs.items():
        assert rt.cudaMemset(o[k], 0, ctypes.c_size_t(n)) == 0
    status = dev_alloc(4)
    assert rt.cudaMemset(status, 0, ctypes.c_size_t(4)) == 0
    r.opt.bwd_stages = 0
    L = lib.load()
    st = L.hm_blend_backward_noalloc(
        r.cams, len(r.cams), r.n, d["means"], d["scales"], d["quats"], d["opacity"], None, d["sh"],
        r.sh_degree, r.sh_format, d["records"], d["pair_vals"], d["ranges"], d["mesh_depth"],
        d["mesh_rgb"], d["uv"], tw, th, ctypes.byref(r.opt), d["T"], d["last_idx"], d["dI"], None,
        None, o["means"], o["scales"], o["quats"], o["opacity"], o["sh"], o["texture"], status, None)
    assert st == 0, lib.last_error()
    assert rt.cudaDeviceSynchronize() == 0
    for k, n in outs.items():
        buf = ctypes.create_string_buffer(n)
        assert rt.cudaMemcpy(buf, o[k], ctypes.c_size_t(n), 2) == 0
        got = np.frombuffer(buf.raw, dtype=np.float32).reshape(want[k].shape)
        tol = 1e-5 * float(np.abs(want[k]).max()) + 1e-12
        assert np.allclose(got, want[k], rtol=1e-5, atol=tol), k
    print("RESET_OK", flush=True)
    os._exit(0)                  # torch's context is gone: skip its teardown
""")


def test_noalloc_finds_its_array_again_after_a_context_reset():
    """Call, cudaDeviceReset, call again (in a child process, since the reset
    ends every allocation of the process): the second call looks the array
    up in the new context and gives the same gradients."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, HM_ROOT=root)
    p = subprocess.run([sys.executable, "-c", _RESET_CHILD], env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0 and "RESET_OK" in p.stdout, p.stdout[-2000:] + p.stderr[-4000:]
