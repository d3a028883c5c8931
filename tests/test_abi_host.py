"""The C-ABI library loads and exports every entry point include/hm.h
declares; host-side logic (options, tile counts, workspace sizes, argument
validation) works without a GPU.  No call here launches a kernel."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2506_06988_b300 import build, lib, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hm():
    build.build()
    return lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "hm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(hm):
    declared = _declared()
    assert len(declared) >= 11
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (hm_[a-z0-9_]+)", out))
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    assert set(lib.EXPORTS) == set(declared)
    for name in declared:
        assert hasattr(hm, name)


def test_library_is_built_for_sm_103a():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getmtime(lib.LIB_PATH) >= max(
        os.path.getmtime(os.path.join(build.CSRC, f)) for f in os.listdir(build.CSRC))


def test_default_options(hm):
    o = lib.HmOptions()
    hm.hm_default_options(ctypes.byref(o))
    assert (o.tile_w, o.tile_h, o.batch, o.mesh_cull, o.ellipse_cull, o.bwd_stages) == (16, 16, 128, 1, 1, 0)
    assert abs(o.near_gauss - 0.2) < 1e-7 and abs(o.near_mesh - 0.01) < 1e-9
    assert list(o.bg) == [0.0, 0.0, 0.0]


def test_total_tiles_and_ragged_sizes(hm):
    cams = [scenes._identity_cam(37, 23), scenes._identity_cam(16, 16), scenes._identity_cam(1, 1)]
    c = lib.cameras(cams)
    for tile, want in (((16, 16), 3 * 2 + 1 + 1), ((32, 8), 2 * 3 + 1 * 2 + 1), ((8, 8), 5 * 3 + 4 + 1)):
        assert lib.hm_total_tiles(c, lib.options(tile=tile)) == want


def test_invalid_arguments_are_rejected_on_the_host(hm):
    cams = lib.cameras([scenes._identity_cam()])
    bad_tile = lib.options(tile=(16, 16))
    bad_tile.tile_w = 12
    assert hm.hm_total_tiles(cams, 1, ctypes.byref(bad_tile)) == -1
    assert "tile shape" in lib.last_error()
    o = lib.options()
    # sh_degree out of range
    st = lib.hm_project_gaussians(cams, 1, 0, 0, 0, 0, 0, 5, lib.HM_SH_F32, o, 0, 0)
    assert st == lib.HM_ERR_INVALID_ARG and "sh_degree" in lib.last_error()
    # too many views
    many = lib.cameras([scenes._identity_cam()] * (lib.HM_MAX_VIEWS + 1))
    st = lib.hm_project_gaussians(many, 1, 0, 0, 0, 0, 0, 0, lib.HM_SH_F32, o, 0, 0)
    assert st == lib.HM_ERR_INVALID_ARG
    # zero-size image
    z = scenes._identity_cam(0, 4)
    st = lib.hm_project_gaussians(lib.cameras([z]), 1, 0, 0, 0, 0, 0, 0, lib.HM_SH_F32, o, 0, 0)
    assert st == lib.HM_ERR_INVALID_ARG and "image size" in lib.last_error()
    # capacity above the 2^30 limit
    st = lib.hm_bin_sort(cams, 1, 0, None, o, 0, lib.HM_MAX_PAIRS + 1, 0, 0, 0, 0, 0, 0)
    assert st == lib.HM_ERR_INVALID_ARG
    # batch larger than the tile
    ob = lib.options(tile=(8, 8))
    ob.batch = 128
    st = lib.hm_blend_forward(cams, 1, 0, 0, 8, 0, 0, ob, 8, 8, 8, 0, None, None, 0)
    assert st == lib.HM_ERR_INVALID_ARG and "batch" in lib.last_error()
    # misaligned records
    st = lib.hm_blend_forward(cams, 10, 4, 8, 8, 0, 0, o, 8, 8, 8, 0, None, None, 0)
    assert st == lib.HM_ERR_INVALID_ARG and "aligned" in lib.last_error()
    # a persistent launch without its work counter
    op = lib.options(persistent=True)
    st = lib.hm_blend_forward(cams, 10, 16, 8, 8, 0, 0, op, 8, 8, 8, 0, None, None, 0)
    assert st == lib.HM_ERR_INVALID_ARG and "work counter" in lib.last_error()
    # workspace too small
    st = lib.hm_bin_sort(cams, 10, 16, None, o, 16, 1000, 16, 16, 0, 16, 8, 0)
    assert st == lib.HM_ERR_WORKSPACE


def test_workspace_sizes_grow_with_the_problem(hm):
    cams = lib.cameras([scenes._identity_cam(64, 48)] * 2)
    o = lib.options()
    a = lib.hm_bin_sort_workspace_size(cams, 1000, 10_000, o)
    b = lib.hm_bin_sort_workspace_size(cams, 2000, 10_000, o)
    c = lib.hm_bin_sort_workspace_size(cams, 1000, 100_000, o)
    assert 0 < a < b and a < c           # per-record list, per-pair and per-tile scratch
    r1 = lib.hm_rasterize_mesh_workspace_size(cams, 100, 200, 5000, o)
    r2 = lib.hm_rasterize_mesh_workspace_size(cams, 100, 200, 50_000, o)
    assert 0 < r1 < r2
    # the replay's nine partials per record, then the list of (Gaussian, view)
    # pairs with a gradient (8 bytes per record)
    assert lib.hm_blend_backward_workspace_size(2, 1000) >= 2 * 1000 * (9 * 4 + 8)
    assert lib.hm_blend_backward_workspace_size(2, 2000) - lib.hm_blend_backward_workspace_size(2, 1000) == \
        2 * 1000 * (9 * 4 + 8)
    # the no-allocation entry point's static scratch holds exactly the problems whose workspace fits
    n_max = 381_294
    assert lib.hm_blend_backward_workspace_size(1, n_max) <= lib.HM_BWD_NOALLOC_BYTES
    assert lib.hm_blend_backward_workspace_size(1, n_max + 1) > lib.HM_BWD_NOALLOC_BYTES


def test_product_package_does_not_import_the_oracle():
    """The CUDA path never routes through the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2506_06988_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower() or f == "scenes.py", f


def test_texture_loss_schedule_follows_the_paper():
    """lambda_t: 0 through the 3k-iteration warm-up, 0.1 strictly between it
    and the end of densification at 15k, 0 afterwards (Sec. 3.4, Sec. 4.1,
    Algorithm 1's strict comparisons)."""
    from paper_2506_06988_b300.schedule import texture_loss_weight
    assert texture_loss_weight(0) == 0.0
    assert texture_loss_weight(3000) == 0.0
    assert texture_loss_weight(3001) == 0.1
    assert texture_loss_weight(14999) == 0.1
    assert texture_loss_weight(15000) == 0.0
    assert texture_loss_weight(30000) == 0.0


def test_loss_defaults_and_invalid_args():
    p = lib.loss_params()
    assert abs(p.lambda_ssim - 0.2) < 1e-7 and abs(p.lambda_t - 0.1) < 1e-7 and p.k == 20.0
    cams = lib.cameras([scenes._identity_cam(16, 16)])
    assert lib.hm_hybrid_loss_workspace_size(cams) >= 9 * 16 * 16 * 4
    st = lib.hm_hybrid_loss(cams, 16, 16, 16, None, None, p, 16, 16, None, 16, 1, 0)
    assert st == lib.HM_ERR_INVALID_ARG and "mesh" in lib.last_error()
    bad = lib.loss_params(lambda_ssim=1.5)
    st = lib.hm_hybrid_loss(cams, 16, 16, None, None, None, bad, 16, 16, None, 16, 1 << 20, 0)
    assert st == lib.HM_ERR_INVALID_ARG
    st = lib.hm_hybrid_loss(cams, 16, 16, None, None, None, p, 16, 16, None, 16, 8, 0)
    assert st == lib.HM_ERR_WORKSPACE


def test_checked_library_exports_the_same_entry_points():
    # libhm_checked.so: the same sources built with HM_CHECKED (index checks
    # that report instead of faulting); the default library has no checks
    build.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_CHECKED_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (hm_[a-z0-9_]+)", out))
    assert not [d for d in _declared() if d not in exported]
    chk = lib.load_checked()
    assert chk is not lib.load()
    v = ctypes.c_int32(7)
    assert lib.load().hm_checked_status(ctypes.byref(v), 0) == lib.HM_ERR_INVALID_ARG
    assert "not the checked build" in lib.last_error() and v.value == 0
    assert chk.hm_checked_status(None, 0) == lib.HM_ERR_INVALID_ARG
