"""Tile shapes (unigs_config.tile_w x tile_h: 16 x 16, 8 x 32, 32 x 8, 64 x 4).

The tile shape decides which (tile, Gaussian) pairs the binning lists - the
keys, values and ranges must match the oracle's float32 recipe for that shape
bit for bit - but not the image: each Gaussian is drawn on the pixels of its
3-sigma square, so every pixel blends the same Gaussians in the same order for
every shape.  On the FP32-pipe path the outputs are therefore bit-identical
across shapes (n_contrib, a position in the tile's list, aside); the
tensor-core logit blend moves by float32 summation order only.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_12174_gb300 import abi
from paper_2510_12174_gb300 import rasterizer as rz
from paper_2510_12174_gb300 import scenes

from gpu_helpers import (MAX_AMBIGUOUS_FWD, MAX_AMBIGUOUS_GRAD, TOL_ABS, TOL_REL,
                         check_grad_errors, flat_upstream, forward_errors, grad_errors,
                         masked_upstream)

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (8, 32), (32, 8), (64, 4)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    torch.cuda.set_device(0)


def _cfg(tile, simt=False):
    cfg = abi.unigs_config_default()
    cfg.tile_w, cfg.tile_h = tile
    if simt:
        cfg.flags |= abi.UNIGS_FLAG_SIMT_LOGITS
    return cfg


def _scene():
    # two cameras of ragged sizes (neither a multiple of 64 nor of 32)
    return scenes.small_room(n=6000, width=100, height=76, n_sem=16, seed=71, n_cams=2)


@pytest.mark.parametrize("tile", SHAPES)
def test_binning_bit_exact_per_shape(tile):
    sc, cams = _scene()
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams, cfg=_cfg(tile))
    r.forward()
    torch.cuda.synchronize()
    assert (int(r.plan.cfg.tile_w), int(r.plan.cfg.tile_h)) == tile
    keys, vals, ranges = r.sorted_instances()
    ref = oracle.bin_cameras_fast(sc, cams, tile)
    assert np.array_equal(keys, ref["keys"]) and np.array_equal(vals, ref["vals"])
    assert np.array_equal(ranges, ref["ranges"])
    assert int(r.plan.n_tiles) == len(ref["ranges"])


@pytest.mark.parametrize("tile", SHAPES[1:])
def test_forward_parity_per_shape(tile):
    sc, cams = _scene()
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams, cfg=_cfg(tile))
    out = r.forward()
    torch.cuda.synchronize()
    _, ref, _ = oracle.render(sc, cams, with_normal_d=False, tile=tile)
    e = forward_errors(r, out, ref, sc.n_sem)
    print(tile, e)
    assert e["ambiguous_fraction"] < MAX_AMBIGUOUS_FWD
    assert e["rgb"] < TOL_ABS and e["normal_g"] < TOL_ABS and e["kmap"] < TOL_ABS
    assert e["T_final"] < TOL_ABS and e["depth"] < TOL_REL and e["logits"] < TOL_REL
    assert e["n_contrib"] == 0


def test_outputs_do_not_depend_on_tile_shape():
    sc, cams = _scene()
    outs = {}
    for tile in SHAPES:
        for simt in (True, False):
            r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams, cfg=_cfg(tile, simt))
            outs[(tile, simt)] = r.forward()
            torch.cuda.synchronize()
    fmax = float(np.abs(sc.sem).max())
    for tile in SHAPES[1:]:
        for simt in (True, False):
            a, b = outs[(tile, simt)], outs[(SHAPES[0], simt)]
            for k in ("rgb", "depth", "normal_g", "kmap", "T_final", "normal_d"):
                assert torch.equal(a[k], b[k]), (tile, simt, k)
            if simt:
                assert torch.equal(a["logits"], b["logits"]), tile
            else:
                assert float((a["logits"] - b["logits"]).abs().max()) < 1e-5 * fmax, tile


def test_backward_parity_at_a_wide_tile():
    sc, cams = scenes.small_room(n=6000, width=64, height=52, n_sem=8, seed=72)
    tile = (32, 8)
    up = scenes.upstream_grads(cams, sc.n_sem, seed=73)
    _, ref_fwd, _ = oracle.render(sc, cams, tile=tile)
    amb = np.mean(np.concatenate([rf["amb_grad"].numpy().ravel() for rf in ref_fwd]))
    assert amb < MAX_AMBIGUOUS_GRAD
    up = masked_upstream(up, [rf["amb_grad"].numpy() for rf in ref_fwd])
    up["normal_d"] = [np.zeros_like(a) for a in up["normal_d"]]
    _, gref, _ = oracle.render_and_grad(sc, cams, up, tile=tile)
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams, cfg=_cfg(tile))
    out = r.forward()
    fu = flat_upstream(up)
    grads = r.backward(out, {k: fu[k] for k in fu if k != "normal_d"})
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    check_grad_errors(grad_errors(grads, gref))


def test_invalid_tile_shape_rejected():
    sc, cams = scenes.small_room(n=100, seed=74)
    for tile in ((16, 8), (32, 16), (4, 64), (16, 0)):
        with pytest.raises(abi.UnigsError):
            rz.Renderer(rz.DeviceScene.from_scene(sc), cams, cfg=_cfg(tile))
