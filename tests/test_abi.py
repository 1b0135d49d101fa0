"""The C-ABI library builds, loads and exports every entry point that
include/unigs.h declares; host-side argument checks (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(unigs_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2510_12174_gb300 import abi
    return abi


def test_header_declares_entry_points():
    names = _declared()
    for n in ("unigs_preprocess", "unigs_bin_sort", "unigs_render_fwd", "unigs_render_bwd",
              "unigs_depth_normal_fwd", "unigs_depth_normal_bwd", "unigs_plan_init",
              "unigs_loss", "unigs_adam_step", "unigs_param_copies", "unigs_prune_mark",
              "unigs_prune_compact", "unigs_sort_pairs_static"):
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
    # (camera, Gaussian) pair indices are 32-bit in the device lists
    arr3 = rz.make_cameras([cams[0]] * 3)
    g.n = 2 ** 31 - 1
    assert lib.unigs_plan_init(plan, g, arr3, 3, None, 0) == lib.UNIGS_ERR_INVALID_ARG
    g.n = 2 ** 31 - 1
    assert lib.unigs_plan_init(plan, g, arr3, 2, None, 0) == lib.UNIGS_OK  # 2^32 - 2 pairs
    g.n = 10
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


def test_training_entry_points_check_arguments_on_host(lib):
    """The training entry points refuse bad arguments before any launch."""
    import ctypes
    from paper_2510_12174_gb300 import rasterizer as rz, scenes
    L = lib.lib()
    lam = lib.unigs_loss_lambda()
    L.unigs_loss_lambda_default(ctypes.byref(lam))
    assert (lam.l1, round(lam.normal, 6), round(lam.depth, 6), round(lam.seg, 6),
            round(lam.K, 6)) == (1.0, 0.1, 0.1, 0.1, 0.1)
    sc, cams = scenes.small_room(n=10, width=20, height=20)
    g = lib.unigs_gaussians()
    g.n, g.sh_degree, g.n_sem, g.feat_dtype = 10, 3, 8, 0
    plan = lib.unigs_plan()
    assert lib.unigs_plan_init(plan, g, rz.make_cameras(cams), 1, None, 0) == lib.UNIGS_OK
    out = lib.unigs_outputs()
    tgt = lib.unigs_targets()
    grads = lib.unigs_loss_grads()
    args = (ctypes.byref(plan), ctypes.byref(out), None, ctypes.byref(tgt), ctypes.byref(lam))
    # no record
    assert L.unigs_loss(*args, 16, None, ctypes.byref(grads), None) == lib.UNIGS_ERR_INVALID_ARG
    # a target without its output
    tgt.rgb = 16
    assert L.unigs_loss(*args, 16, 16, ctypes.byref(grads), None) == lib.UNIGS_ERR_INVALID_ARG
    tgt.rgb = None
    tgt.normal = 16                      # normal target without the normal-from-depth map
    assert L.unigs_loss(*args, 16, 16, ctypes.byref(grads), None) == lib.UNIGS_ERR_INVALID_ARG
    # Adam: too many groups, a bad activation, an activated copy over the raw values
    hp = lib.unigs_adam_hparams(0.9, 0.999, 1e-15)
    groups = (lib.unigs_adam_group * 1)()
    assert L.unigs_adam_step(groups, 17, ctypes.byref(hp), 16, None) == lib.UNIGS_ERR_INVALID_ARG
    G = groups[0]
    G.param, G.grad, G.m, G.v, G.count = 16, 32, 48, 64, 4
    G.activation = 3
    assert L.unigs_adam_step(groups, 1, ctypes.byref(hp), 16, None) == lib.UNIGS_ERR_INVALID_ARG
    G.activation = lib.UNIGS_ACT_EXP
    G.act_out = 16
    assert L.unigs_adam_step(groups, 1, ctypes.byref(hp), 16, None) == lib.UNIGS_ERR_INVALID_ARG
    assert L.unigs_param_copies(groups, 1, None) == lib.UNIGS_ERR_INVALID_ARG
    G.act_out, G.m = None, None          # missing moment
    assert L.unigs_adam_step(groups, 1, ctypes.byref(hp), 16, None) == lib.UNIGS_ERR_INVALID_ARG
    assert L.unigs_adam_step(groups, 1, ctypes.byref(hp), None, None) == lib.UNIGS_ERR_INVALID_ARG
    # pruning: workspace size grows with n; bad sizes, aliasing, fill of 2-byte elements
    assert L.unigs_prune_workspace_bytes(1000) > L.unigs_prune_workspace_bytes(10) > 0
    nk = ctypes.c_int64(0)
    assert L.unigs_prune_mark(16, -1, 0.2, 16, ctypes.byref(nk), None) == lib.UNIGS_ERR_INVALID_ARG
    assert L.unigs_prune_mark(16, 10, 0.2, 8, ctypes.byref(nk), None) == lib.UNIGS_ERR_INVALID_ARG
    arr = (lib.unigs_prune_array * 1)()
    arr[0].src, arr[0].dst, arr[0].planes, arr[0].row, arr[0].elem_bytes = 16, 16, 1, 1, 4
    assert L.unigs_prune_compact(arr, 1, 10, 5, 16, None) == lib.UNIGS_ERR_INVALID_ARG
    arr[0].dst, arr[0].elem_bytes, arr[0].fill = 32, 2, 1
    assert L.unigs_prune_compact(arr, 1, 10, 5, 16, None) == lib.UNIGS_ERR_INVALID_ARG
    arr[0].elem_bytes, arr[0].fill = 4, 0
    assert L.unigs_prune_compact(arr, 1, 10, 11, 16, None) == lib.UNIGS_ERR_INVALID_ARG


def test_launch_shape_fields_are_validated(lib):
    from paper_2510_12174_gb300 import rasterizer as rz, scenes
    sc, cams = scenes.small_room(n=10, width=20, height=20)
    g = lib.unigs_gaussians()
    g.n, g.sh_degree, g.n_sem, g.feat_dtype = 10, 3, 8, 1
    plan = lib.unigs_plan()
    arr = rz.make_cameras(cams)
    for field, value, ok in (("batch", 8, True), ("batch", 48, False), ("batch_fwd", 8, False),
                             ("batch_fwd", 64, True), ("ctas_per_sm", 9, False),
                             ("ctas_per_sm_fwd", 4, True), ("flags", 8, False), ("flags", 4, True),
                             ("flags", 7, True), ("alpha_max", 1.0, False),
                             ("alpha_max", 0.999, True), ("alpha_max", float("nan"), False),
                             ("alpha_min", -1e-3, False), ("alpha_min", 0.995, False),
                             ("T_min", 1.0, False), ("lowpass", float("inf"), False)):
        cfg = lib.unigs_config_default()
        setattr(cfg, field, value)
        want = lib.UNIGS_OK if ok else lib.UNIGS_ERR_INVALID_ARG
        assert lib.unigs_plan_init(plan, g, arr, 1, cfg, 0) == want, (field, value)


def test_plan_paths_select_the_composite_kernels(lib):
    """unigs_plan_paths: which composites a plan runs, decided on the host from
    the logit width, the feature dtype, the SIMT flag and the launch shapes;
    the float32 logit copy (and its workspace) only where an FP32-pipe
    composite reads bfloat16 rows."""
    from paper_2510_12174_gb300 import rasterizer as rz, scenes
    sc, cams = scenes.small_room(n=10, width=20, height=20)
    arr = rz.make_cameras(cams)
    FWD, BWD, S32 = lib.UNIGS_PATH_FWD_TC, lib.UNIGS_PATH_BWD_TC, lib.UNIGS_PATH_SEM32

    def paths(n_sem, bf16, flags=0, batch=0, ctas=0):
        g = lib.unigs_gaussians()
        g.n, g.sh_degree, g.n_sem, g.feat_dtype = 1000, 3, n_sem, 1 if bf16 else 0
        cfg = lib.unigs_config_default()
        cfg.flags |= flags
        cfg.batch, cfg.ctas_per_sm = batch, ctas
        plan = lib.unigs_plan()
        assert lib.unigs_plan_init(plan, g, arr, 1, cfg, 0) == lib.UNIGS_OK
        return lib.unigs_plan_paths(plan), plan.ws_bytes

    p, ws_tc = paths(64, True)
    assert p == FWD | BWD
    p, ws_simt = paths(64, True, batch=8, ctas=3)
    assert p == FWD | S32
    assert ws_simt - ws_tc >= 4 * 1000 * 64  # the float32 copy of the rows
    assert paths(64, True, batch=16, ctas=2)[0] == FWD | BWD
    assert paths(64, True, batch=16, ctas=3)[0] == FWD | S32
    assert paths(64, True, flags=lib.UNIGS_FLAG_SIMT_LOGITS)[0] == S32
    assert paths(64, False)[0] == FWD
    assert paths(9, True)[0] == FWD | BWD
    assert paths(8, True)[0] == S32
    assert paths(0, True)[0] == 0
    assert lib.lib().unigs_plan_paths(None) == 0
