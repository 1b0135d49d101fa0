"""FP64 CPU oracle of the UniGS multimodal rasterizer.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow definition that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library never does,
and it imports nothing from the library.  Inputs come from the seeded scene
generator, which holds none of the method's arithmetic.

* :mod:`oracle.binning` - the float32 recipe that decides the tile lists
  (bit-exact target for the GPU's keys, values and ranges).
* :mod:`oracle.raster` - float64 forward (Alg. 2, Eqs. depth_render, t_render,
  semantic_render, the ray-ellipsoid midpoint depth and Alg. 1) whose exact
  derivative autograd takes (the target of Alg. 3, Alg. 4 and the
  preprocess backward).
* :mod:`oracle.sh` - real SH basis to degree 3.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from .binning import bin_cameras, bin_cameras_fast, project_fp32
from .raster import (Bands, Params, Prep, composite_tile, depth_to_normal,
                     preprocess, render_camera)

OUT_KEYS = ("rgb", "depth", "normal", "kmap", "logits", "T")
PARAM_KEYS = ("mean", "quat", "scale", "opacity", "kfac", "sh", "sem")


def render(scene, cams, requires_grad: bool = False, binning=None,
           tiles: Optional[Sequence[Sequence[int]]] = None,
           bands: Optional[Bands] = None, with_normal_d: bool = True,
           center_depth: bool = False, tile=(16, 16)):
    """Forward over all cameras.  Returns (params, per-camera outputs, binning).
    ``tile`` = (TW, TH) is the tile shape of the binning when none is given."""
    if binning is None:
        binning = bin_cameras_fast(scene, cams, tile)
    params = Params.from_scene(scene, requires_grad)
    outs = []
    ctx = torch.enable_grad() if requires_grad else torch.no_grad()
    with ctx:
        for k, cam in enumerate(cams):
            prep = preprocess(params, cam)
            r = render_camera(prep, cam, binning, k,
                              tiles=None if tiles is None else tiles[k], bands=bands,
                              center_depth=center_depth)
            if with_normal_d:
                nd = depth_to_normal(r["depth"], cam)
                r["normal_d"] = nd["normal"]
                r["nd_valid"] = nd["valid"]
                r["nd_amb"] = nd["amb"]
            outs.append(r)
    return params, outs, binning


def render_and_grad(scene, cams, upstream: Dict[str, List[np.ndarray]],
                    binning=None, bands: Optional[Bands] = None, center_depth: bool = False,
                    tiles: Optional[Sequence[Sequence[int]]] = None, tile=(16, 16)):
    """Forward plus exact gradients of L = sum_c <output_c, upstream_c>.

    ``upstream`` maps rgb, depth, normal_g, kmap, logits, normal_d to per-camera
    arrays (as produced by the scene generator).  Returns (outputs, grads) with
    grads keyed like the Gaussian parameters.
    """
    params, outs, binning = render(scene, cams, requires_grad=True, binning=binning,
                                   bands=bands, center_depth=center_depth, tiles=tiles,
                                   tile=tile)
    loss = torch.zeros((), dtype=torch.float64)
    name = {"rgb": "rgb", "depth": "depth", "normal_g": "normal", "kmap": "kmap",
            "logits": "logits", "normal_d": "normal_d"}
    for k, r in enumerate(outs):
        for up, key in name.items():
            g = torch.as_tensor(np.asarray(upstream[up][k], dtype=np.float64))
            loss = loss + (r[key] * g).sum()
    loss.backward()
    grads = {}
    for key, leaf in zip(PARAM_KEYS, params.leaves()):
        grads[key] = (leaf.grad if leaf.grad is not None
                      else torch.zeros_like(leaf)).numpy()
    outs_np = [{k: (v.detach().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
               for r in outs]
    return outs_np, grads, binning


__all__ = ["Bands", "Params", "Prep", "bin_cameras", "bin_cameras_fast",
           "composite_tile", "depth_to_normal", "preprocess", "project_fp32",
           "render", "render_and_grad", "render_camera"]
