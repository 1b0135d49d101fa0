"""ctypes binding of the libunigs C ABI (include/unigs.h, include/unigs_train.h,
include/unigs_anchors.h).

Argument marshalling only: every function here forwards to the entry point
of the same name; all arithmetic runs in the library's kernels.  Loading
fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_float, c_int32, c_int64, c_size_t,
                    c_uint32, c_void_p)

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libunigs.so")

UNIGS_MAX_CAMS = 64
UNIGS_TILE = 16
UNIGS_TILE_PIXELS = 256
TILE_SHAPES = ((16, 16), (8, 32), (32, 8), (64, 4))
UNIGS_MAX_SEM = 64
UNIGS_FLAG_CENTER_DEPTH = 1
UNIGS_FLAG_SIMT_LOGITS = 2
UNIGS_FLAG_CHECK_FINITE = 4
UNIGS_PATH_FWD_TC = 1
UNIGS_PATH_BWD_TC = 2
UNIGS_PATH_SEM32 = 4
UNIGS_STATIC_SORT_MAX_PAIRS = 1 << 20

UNIGS_OK = 0
UNIGS_ERR_INVALID_ARG = 1
UNIGS_ERR_CAPACITY = 2
UNIGS_ERR_CUDA = 3
UNIGS_ERR_NONFINITE = 4
UNIGS_ERR_TIMEOUT = 5


class unigs_camera(Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float), ("R_wc", c_float * 9), ("t_wc", c_float * 3),
                ("R_cw", c_float * 9), ("C", c_float * 3), ("z_near", c_float)]


class unigs_gaussians(Structure):
    _fields_ = [("n", c_int64), ("sh_degree", c_int32), ("n_sem", c_int32),
                ("feat_dtype", c_int32), ("reserved", c_int32), ("mean", c_void_p),
                ("quat", c_void_p), ("scale", c_void_p), ("opacity", c_void_p),
                ("kfac", c_void_p), ("sh", c_void_p), ("sem", c_void_p)]


class unigs_outputs(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("normal_g", c_void_p),
                ("kmap", c_void_p), ("logits", c_void_p), ("T_final", c_void_p),
                ("n_contrib", c_void_p)]


class unigs_grad_outputs(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("normal_g", c_void_p),
                ("kmap", c_void_p), ("logits", c_void_p)]


class unigs_param_grads(Structure):
    _fields_ = [("mean", c_void_p), ("quat", c_void_p), ("scale", c_void_p),
                ("opacity", c_void_p), ("kfac", c_void_p), ("sh", c_void_p),
                ("sem", c_void_p), ("accumulate", c_int32), ("reserved", c_int32)]


class unigs_config(Structure):
    _fields_ = [("alpha_min", c_float), ("alpha_max", c_float), ("T_min", c_float),
                ("lowpass", c_float), ("step1", c_int32), ("step2", c_int32),
                ("lambda_", c_float), ("flags", c_uint32), ("batch", c_int32),
                ("ctas_per_sm", c_int32), ("batch_fwd", c_int32), ("ctas_per_sm_fwd", c_int32),
                ("tile_w", c_int32), ("tile_h", c_int32)]


class unigs_plan(Structure):
    _fields_ = [("n", c_int64), ("n_cams", c_int32), ("n_sem", c_int32),
                ("sh_degree", c_int32), ("feat_dtype", c_int32), ("capacity", c_int64),
                ("n_tiles", c_int64), ("n_pixels", c_int64),
                ("tile_offset", c_int32 * (UNIGS_MAX_CAMS + 1)),
                ("pixel_offset", c_int64 * (UNIGS_MAX_CAMS + 1)),
                ("sort_passes", c_int32), ("reserved", c_int32), ("ws_bytes", c_size_t),
                ("off", c_size_t * 20), ("cfg", unigs_config)]


class unigs_targets(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("normal", c_void_p),
                ("label", c_void_p)]


class unigs_loss_lambda(Structure):
    _fields_ = [("l1", c_float), ("normal", c_float), ("depth", c_float), ("seg", c_float),
                ("K", c_float)]


class unigs_loss_grads(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("normal_d", c_void_p),
                ("kmap", c_void_p), ("logits", c_void_p)]


class unigs_adam_group(Structure):
    _fields_ = [("param", c_void_p), ("grad", c_void_p), ("m", c_void_p), ("v", c_void_p),
                ("act_out", c_void_p), ("bf16_out", c_void_p), ("count", c_int64),
                ("lr", c_float), ("activation", c_int32)]


class unigs_adam_hparams(Structure):
    _fields_ = [("beta1", c_float), ("beta2", c_float), ("eps", c_float)]


class unigs_prune_array(Structure):
    _fields_ = [("src", c_void_p), ("dst", c_void_p), ("planes", c_int32), ("row", c_int32),
                ("elem_bytes", c_int32), ("fill", c_int32), ("fill_value", c_float),
                ("reserved", c_int32)]


UNIGS_ANCHOR_FEAT = 32
UNIGS_ANCHOR_HIDDEN = 32
UNIGS_ANCHOR_MAX_OFFSETS = 16
ANCHOR_MLPS = ("sem", "k", "opacity", "color", "cov")


class unigs_mlp(Structure):
    _fields_ = [("w1", c_void_p), ("b1", c_void_p), ("w2", c_void_p), ("b2", c_void_p)]


class unigs_anchors(Structure):
    _fields_ = [("n", c_int64), ("n_offsets", c_int32), ("feat_dim", c_int32),
                ("hidden", c_int32), ("n_sem", c_int32), ("pos", c_void_p), ("scale", c_void_p),
                ("offsets", c_void_p), ("feat", c_void_p), ("sem", c_void_p),
                ("kfac", c_void_p)] + [("mlp_" + n, unigs_mlp) for n in ANCHOR_MLPS]


class unigs_anchor_gaussians(Structure):
    _fields_ = [("mean", c_void_p), ("quat", c_void_p), ("scale", c_void_p),
                ("opacity", c_void_p), ("kfac", c_void_p), ("sh", c_void_p), ("sem", c_void_p),
                ("feat_dtype", c_int32), ("reserved", c_int32)]


class unigs_mlp_grads(Structure):
    _fields_ = [("w1", c_void_p), ("b1", c_void_p), ("w2", c_void_p), ("b2", c_void_p)]


class unigs_anchor_grads(Structure):
    _fields_ = [("pos", c_void_p), ("scale", c_void_p), ("offsets", c_void_p),
                ("feat", c_void_p), ("sem", c_void_p), ("kfac", c_void_p)] + \
               [("mlp_" + n, unigs_mlp_grads) for n in ANCHOR_MLPS] + \
               [("accumulate", c_int32), ("reserved", c_int32)]


UNIGS_LOSS_TOTAL, UNIGS_LOSS_L1, UNIGS_LOSS_NORMAL, UNIGS_LOSS_DEPTH = 0, 1, 2, 3
UNIGS_LOSS_SEG, UNIGS_LOSS_K = 4, 5
UNIGS_LOSS_W_L1, UNIGS_LOSS_W_NORMAL, UNIGS_LOSS_W_DEPTH = 6, 7, 8
UNIGS_LOSS_W_SEG, UNIGS_LOSS_W_K = 9, 10
UNIGS_LOSS_N_DEPTH, UNIGS_LOSS_N_LABEL = 11, 12
UNIGS_LOSS_RECORD_FLOATS = 16
UNIGS_ACT_NONE, UNIGS_ACT_EXP, UNIGS_ACT_SIGMOID = 0, 1, 2
UNIGS_ADAM_MAX_GROUPS = 16

_lib = None

# (name, restype, argtypes)
_SIGS = [
    ("unigs_config_default", None, [POINTER(unigs_config)]),
    ("unigs_plan_init", c_int32, [POINTER(unigs_plan), POINTER(unigs_gaussians),
                                  POINTER(unigs_camera), c_int32, POINTER(unigs_config), c_int64]),
    ("unigs_workspace_bytes", c_size_t, [POINTER(unigs_plan)]),
    ("unigs_preprocess", c_int32, [POINTER(unigs_plan), POINTER(unigs_gaussians),
                                   POINTER(unigs_camera), c_void_p, c_void_p]),
    ("unigs_bin_sort", c_int32, [POINTER(unigs_plan), c_void_p, POINTER(c_int64), c_void_p]),
    ("unigs_render_fwd", c_int32, [POINTER(unigs_plan), POINTER(unigs_gaussians), c_void_p,
                                   POINTER(unigs_outputs), c_void_p]),
    ("unigs_depth_normal_fwd", c_int32, [POINTER(unigs_plan), POINTER(unigs_camera), c_void_p,
                                         c_void_p, c_void_p]),
    ("unigs_depth_normal_bwd", c_int32, [POINTER(unigs_plan), POINTER(unigs_camera), c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p]),
    ("unigs_render_bwd", c_int32, [POINTER(unigs_plan), POINTER(unigs_gaussians),
                                   POINTER(unigs_camera), c_void_p, POINTER(unigs_outputs),
                                   POINTER(unigs_grad_outputs), POINTER(unigs_param_grads),
                                   c_void_p]),
    ("unigs_status_poll", c_int32, [POINTER(unigs_plan), c_void_p, POINTER(c_int64), c_void_p]),
    ("unigs_stats_poll", c_int32, [POINTER(unigs_plan), c_void_p, POINTER(c_int64),
                                   POINTER(c_int64), c_void_p]),
    ("unigs_launches_per_step", c_int32, [POINTER(unigs_plan)]),
    ("unigs_plan_paths", c_int32, [POINTER(unigs_plan)]),
    ("unigs_status_string", c_char_p, [c_int32]),
    ("unigs_sort_pairs_static", c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_void_p,
                                          c_void_p, c_void_p]),
    ("unigs_probe_fma_sink_floats", c_int64, []),
    ("unigs_probe_fma", c_int32, [c_void_p, c_int32, c_int32, POINTER(c_int64), c_void_p]),
    # include/unigs_train.h
    ("unigs_loss_lambda_default", None, [POINTER(unigs_loss_lambda)]),
    ("unigs_loss", c_int32, [POINTER(unigs_plan), POINTER(unigs_outputs), c_void_p,
                             POINTER(unigs_targets), POINTER(unigs_loss_lambda), c_void_p,
                             c_void_p, POINTER(unigs_loss_grads), c_void_p]),
    ("unigs_adam_step", c_int32, [POINTER(unigs_adam_group), c_int32,
                                  POINTER(unigs_adam_hparams), c_void_p, c_void_p]),
    ("unigs_param_copies", c_int32, [POINTER(unigs_adam_group), c_int32, c_void_p]),
    ("unigs_prune_workspace_bytes", c_size_t, [c_int64]),
    ("unigs_prune_mark", c_int32, [c_void_p, c_int64, c_float, c_void_p, POINTER(c_int64),
                                   c_void_p]),
    ("unigs_prune_compact", c_int32, [POINTER(unigs_prune_array), c_int32, c_int64, c_int64,
                                      c_void_p, c_void_p]),
    # include/unigs_anchors.h
    ("unigs_anchor_decode", c_int32, [POINTER(unigs_anchors), POINTER(unigs_anchor_gaussians),
                                      c_void_p]),
    ("unigs_anchor_decode_bwd", c_int32, [POINTER(unigs_anchors), POINTER(unigs_param_grads),
                                          POINTER(unigs_anchor_grads), c_void_p]),
]


def exported_symbols():
    """Names of the entry points declared in include/*.h."""
    return [s[0] for s in _SIGS]


def lib():
    """The loaded libunigs (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libunigs.so is not built ({LIB_PATH}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class UnigsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = lib().unigs_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)
        self.status = status


def check(status: int, what: str = ""):
    if status != UNIGS_OK:
        raise UnigsError(status, what)


# Thin wrappers with the C names ---------------------------------------------
def unigs_config_default() -> unigs_config:
    c = unigs_config()
    lib().unigs_config_default(ctypes.byref(c))
    return c


def unigs_plan_init(plan, g, cams, n_cams, cfg, capacity) -> int:
    return lib().unigs_plan_init(ctypes.byref(plan), ctypes.byref(g), cams, n_cams,
                                 ctypes.byref(cfg) if cfg is not None else None, capacity)


def unigs_workspace_bytes(plan) -> int:
    return lib().unigs_workspace_bytes(ctypes.byref(plan))


def unigs_preprocess(plan, g, cams, ws, stream) -> int:
    return lib().unigs_preprocess(ctypes.byref(plan), ctypes.byref(g), cams, ws, stream)


def unigs_bin_sort(plan, ws, n_out, stream) -> int:
    return lib().unigs_bin_sort(ctypes.byref(plan), ws,
                                ctypes.byref(n_out) if n_out is not None else None, stream)


def unigs_render_fwd(plan, g, ws, out, stream) -> int:
    return lib().unigs_render_fwd(ctypes.byref(plan), ctypes.byref(g), ws, ctypes.byref(out),
                                  stream)


def unigs_depth_normal_fwd(plan, cams, depth, normal_d, stream) -> int:
    return lib().unigs_depth_normal_fwd(ctypes.byref(plan), cams, depth, normal_d, stream)


def unigs_depth_normal_bwd(plan, cams, depth, g_normal_d, g_depth_in, g_depth_out,
                           stream) -> int:
    return lib().unigs_depth_normal_bwd(ctypes.byref(plan), cams, depth, g_normal_d,
                                        g_depth_in, g_depth_out, stream)


def unigs_render_bwd(plan, g, cams, ws, fwd, grad_out, grads, stream) -> int:
    return lib().unigs_render_bwd(ctypes.byref(plan), ctypes.byref(g), cams, ws,
                                  ctypes.byref(fwd), ctypes.byref(grad_out),
                                  ctypes.byref(grads), stream)


def unigs_status_poll(plan, ws, detail, stream) -> int:
    return lib().unigs_status_poll(ctypes.byref(plan), ws,
                                   ctypes.byref(detail) if detail is not None else None, stream)


def unigs_stats_poll(plan, ws, n_eval, n_blend, stream) -> int:
    return lib().unigs_stats_poll(ctypes.byref(plan), ws, ctypes.byref(n_eval),
                                  ctypes.byref(n_blend), stream)


def unigs_sort_pairs_static(keys_in, vals_in, n, key_bits, keys_out, vals_out, stream) -> int:
    """Allocation-free stable radix sort of (u64 key, u32 value) pairs by the
    low ``key_bits`` bits; device pointers; scratch is the library's static
    array (see include/unigs.h)."""
    return lib().unigs_sort_pairs_static(keys_in, vals_in, n, key_bits, keys_out, vals_out,
                                         stream)


def unigs_probe_fma_sink_floats() -> int:
    return lib().unigs_probe_fma_sink_floats()


def unigs_probe_fma(sink, iters, packed, flops_out, stream) -> int:
    """FP32 FMA throughput probe (measurement utility, include/unigs.h)."""
    return lib().unigs_probe_fma(sink, iters, packed, flops_out, stream)


def unigs_launches_per_step(plan) -> int:
    return lib().unigs_launches_per_step(ctypes.byref(plan))


def unigs_plan_paths(plan) -> int:
    return lib().unigs_plan_paths(ctypes.byref(plan))


# include/unigs_train.h ---------------------------------------------------------
def unigs_loss_lambda_default() -> unigs_loss_lambda:
    lam = unigs_loss_lambda()
    lib().unigs_loss_lambda_default(ctypes.byref(lam))
    return lam


def unigs_loss(plan, out, normal_d, tgt, lam, ws, record, grads, stream) -> int:
    """Combined loss of Sec. 3.4 and its gradients (see include/unigs_train.h)."""
    return lib().unigs_loss(ctypes.byref(plan), ctypes.byref(out), normal_d, ctypes.byref(tgt),
                            ctypes.byref(lam), ws, record, ctypes.byref(grads), stream)


def unigs_adam_step(groups, n_groups, hp, step, stream) -> int:
    return lib().unigs_adam_step(groups, n_groups, ctypes.byref(hp), step, stream)


def unigs_param_copies(groups, n_groups, stream) -> int:
    return lib().unigs_param_copies(groups, n_groups, stream)


def unigs_prune_workspace_bytes(n) -> int:
    return lib().unigs_prune_workspace_bytes(n)


def unigs_prune_mark(k, n, T_k, ws, n_keep, stream) -> int:
    return lib().unigs_prune_mark(k, n, T_k, ws, ctypes.byref(n_keep), stream)


def unigs_prune_compact(arrays, n_arrays, n, n_keep, ws, stream) -> int:
    return lib().unigs_prune_compact(arrays, n_arrays, n, n_keep, ws, stream)


def unigs_anchor_decode(a, out, stream) -> int:
    return lib().unigs_anchor_decode(ctypes.byref(a), ctypes.byref(out), stream)


def unigs_anchor_decode_bwd(a, g, out, stream) -> int:
    return lib().unigs_anchor_decode_bwd(ctypes.byref(a), ctypes.byref(g), ctypes.byref(out),
                                         stream)
