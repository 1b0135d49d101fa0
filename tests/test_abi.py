"""The C-ABI library builds, loads and exports every entry point that
include/unigs.h declares; host-side argument checks (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "unigs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(unigs_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2510_12174_gb300 import abi
    return abi


def test_header_declares_entry_points():
    names = _declared()
    for n in ("unigs_preprocess", "unigs_bin_sort", "unigs_render_fwd", "unigs_render_bwd",
              "unigs_depth_normal_fwd", "unigs_depth_normal_bwd", "unigs_plan_init"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    for n in _declared():
        assert hasattr(L, n), n
    assert set(_declared()) <= set(lib.exported_symbols()) | {"unigs_status_string"}


def test_plan_rejects_bad_arguments_on_host(lib):
    from paper_2510_12174_gb300 import rasterizer as rz, scenes
    sc, cams = scenes.small_room(n=10, width=20, height=20)
    g = lib.unigs_gaussians()
    g.n, g.sh_degree, g.n_sem, g.feat_dtype = 10, 3, 8, 0
    arr = rz.make_cameras(cams)
    plan = lib.unigs_plan()
    assert lib.unigs_plan_init(plan, g, arr, 1, None, 0) == lib.UNIGS_OK
    assert plan.ws_bytes > 0 and plan.n_tiles == 4 and plan.n_pixels == 400
    assert plan.sort_passes == 5  # 32 depth bits + 2 tile bits
    g.sh_degree = 4
    assert lib.unigs_plan_init(plan, g, arr, 1, None, 0) == lib.UNIGS_ERR_INVALID_ARG
    g.sh_degree = 3
    assert lib.unigs_plan_init(plan, g, arr, 0, None, 0) == lib.UNIGS_ERR_INVALID_ARG
    g.n_sem = 65
    assert lib.unigs_plan_init(plan, g, arr, 1, None, 0) == lib.UNIGS_ERR_INVALID_ARG
    g.n_sem = 8
    cfg = lib.unigs_config_default()
    cfg.step1 = 5
    assert lib.unigs_plan_init(plan, g, arr, 1, cfg, 0) == lib.UNIGS_ERR_INVALID_ARG
    bad = rz.make_cameras(cams)
    bad[0].width = 0
    assert lib.unigs_plan_init(plan, g, bad, 1, None, 0) == lib.UNIGS_ERR_INVALID_ARG
    # entry points reject NULL / mismatched arguments before touching the GPU
    assert lib.unigs_plan_init(plan, g, arr, 1, None, 0) == lib.UNIGS_OK
    assert lib.unigs_preprocess(plan, g, arr, None, None) == lib.UNIGS_ERR_INVALID_ARG
    assert lib.unigs_bin_sort(plan, None, None, None) == lib.UNIGS_ERR_INVALID_ARG
    out = lib.unigs_outputs()
    assert lib.unigs_render_fwd(plan, g, None, out, None) == lib.UNIGS_ERR_INVALID_ARG
    assert lib.lib().unigs_status_string(2) == b"instance capacity exceeded"


def test_multi_camera_plan_offsets(lib):
    from paper_2510_12174_gb300 import rasterizer as rz, scenes
    cams = scenes.orbit_cameras(3, seed=1, resolutions=[(640, 480), (1280, 720), (1920, 1080)])
    g = lib.unigs_gaussians()
    g.n, g.sh_degree, g.n_sem, g.feat_dtype = 100, 3, 64, 1
    plan = lib.unigs_plan()
    assert lib.unigs_plan_init(plan, g, rz.make_cameras(cams), 3, None, 0) == lib.UNIGS_OK
    t = [40 * 30, 80 * 45, 120 * 68]
    assert list(plan.tile_offset[:4]) == [0, t[0], t[0] + t[1], sum(t)]
    assert list(plan.pixel_offset[:4]) == [0, 307200, 307200 + 921600, 307200 + 921600 + 2073600]
    assert plan.capacity == 4 * 100 * 3
