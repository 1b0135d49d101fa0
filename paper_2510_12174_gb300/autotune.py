"""Launch-shape autotuner for the two composite kernels.

The composites (forward Alg. 2 and backward Alg. 4) are persistent kernels
whose CTAs pull 16x16 tiles from a device work counter, longest Gaussian list
first.  Two launch parameters change their speed but not their results:

* ``batch``: Gaussians staged per shared-memory batch (16, 32 or 64).  Larger
  batches amortise the barrier and bulk-copy issue per Gaussian; smaller ones
  waste less of the last batch of short lists.
* ``ctas_per_sm``: resident persistent CTAs per SM (1-3).  More CTAs hide the
  barrier and atomic latency of the backward; fewer leave more shared memory
  per CTA (the backward's 64-logit, batch-64 stage needs ~123 KB).

The forward output is bit-identical for every shape (each pixel blends its
list in the same order); the gradients differ only in the order of float32
atomic additions.  The tile itself stays 16x16 pixels: it is the binning unit
whose keys and ranges the library reproduces bit for bit, so it is not a
tuning knob.

:func:`tune` times forward + backward of each candidate on the caller's scene
and cameras with CUDA events and keeps the fastest; results are cached in a
JSON file keyed by :func:`workload_key` (GPU, SM count, logit class, feature
dtype, camera count and pixel/Gaussian magnitudes), so a training run pays the
search once per workload class.  :func:`config_for` returns a
``unigs_config`` with the cached shape (or the library default).
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, Optional, Sequence, Tuple

import torch

from . import abi
from . import rasterizer as rz

CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (32, 2), (16, 2), (64, 1), (64, 2), (32, 1), (32, 3), (16, 3))


def default_cache_path() -> str:
    p = os.environ.get("UNIGS_TUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "unigs_gb300", "launch_shapes.json")


def _logit_class(n_sem: int) -> int:
    """The kernels' compiled logit width: 8, 16, 32 or 64 (0 without logits)."""
    if n_sem <= 0:
        return 0
    for c in (8, 16, 32):
        if n_sem <= c:
            return c
    return 64


def key_for(gpu_name: str, sm_count: int, n_sem: int, feat_dtype: str,
            cam_sizes: Sequence[Tuple[int, int]], n_gaussians: int) -> str:
    """Cache key of a workload class: GPU, SM count, compiled logit width,
    feature dtype, camera count, and the pixel and Gaussian counts rounded to
    powers of two."""
    pixels = sum(int(w) * int(h) for w, h in cam_sizes)
    return (f"{gpu_name}|sm{int(sm_count)}|sem{_logit_class(n_sem)}|{feat_dtype}|"
            f"cams{len(cam_sizes)}|px2^{round(math.log2(max(pixels, 1)))}|"
            f"n2^{round(math.log2(max(int(n_gaussians), 1)))}")


def workload_key(scene: "rz.DeviceScene", cams: Sequence, device=None) -> str:
    dev = torch.device(device if device is not None else scene.mean.device)
    props = torch.cuda.get_device_properties(dev)
    dtype = "bf16" if scene.sh.dtype == torch.bfloat16 else "f32"
    return key_for(props.name, props.multi_processor_count, scene.n_sem, dtype,
                   [(c.width, c.height) for c in cams], int(scene.mean.shape[-1]))


def _load(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _store(path: str, key: str, entry: dict) -> None:
    d = _load(path)
    d[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def make_config(batch: int, ctas_per_sm: int, base: Optional[abi.unigs_config] = None):
    cfg = (abi.unigs_config.from_buffer_copy(base) if base is not None
           else abi.unigs_config_default())
    cfg.batch, cfg.ctas_per_sm = int(batch), int(ctas_per_sm)
    return cfg


def _synthetic_upstream(r: "rz.Renderer", seed: int) -> Dict[str, torch.Tensor]:
    g = torch.Generator(device=r.device).manual_seed(seed)
    P = r.n_pixels
    f = lambda c: torch.randn(c * P, generator=g, device=r.device)
    up = {"rgb": f(3), "depth": f(1), "normal_g": f(3), "kmap": f(1)}
    up["logits"] = f(r.scene.n_sem) if r.scene.n_sem else None
    return up


def time_shape(scene, cams, batch: int, ctas_per_sm: int, reps: int = 3,
               base: Optional[abi.unigs_config] = None, seed: int = 0) -> float:
    """Milliseconds of one forward (preprocess, sort, composite) + backward at
    the given launch shape, median of ``reps`` after one warm-up."""
    r = rz.Renderer(scene, cams, cfg=make_config(batch, ctas_per_sm, base))
    out = r.forward()                       # sizes the instance capacity
    up = _synthetic_upstream(r, seed)
    grads = r.alloc_grads()
    stream = torch.cuda.current_stream(r.device)
    r.backward(out, up, grads=grads)
    times = []
    for _ in range(max(1, reps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.forward(out, readback=False, normal_d=False)
        r.backward(out, up, grads=grads)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    s, need = r.status()
    abi.check(s, f"launch shape ({batch}, {ctas_per_sm})")
    times.sort()
    return times[len(times) // 2]


def tune(scene, cams, candidates: Iterable[Tuple[int, int]] = CANDIDATES, reps: int = 3,
         base: Optional[abi.unigs_config] = None, cache_path: Optional[str] = None,
         force: bool = False, timer=None) -> Tuple[int, int]:
    """Fastest (batch, ctas_per_sm) for this scene and camera set; cached.

    ``timer(batch, ctas_per_sm) -> ms`` replaces the CUDA-event timing of
    :func:`time_shape` (for callers with their own step to time)."""
    path = cache_path or default_cache_path()
    key = workload_key(scene, cams)
    return search(key, candidates, path, force,
                  timer or (lambda b, c: time_shape(scene, cams, b, c, reps=reps, base=base)))


def search(key: str, candidates: Iterable[Tuple[int, int]], path: str, force: bool,
           timer) -> Tuple[int, int]:
    """Cache lookup, else time every candidate and store the fastest."""
    if not force:
        hit = _load(path).get(key)
        if hit:
            return int(hit["batch"]), int(hit["ctas_per_sm"])
    results = {}
    for b, c in candidates:
        if b not in (16, 32, 64) or not 1 <= c <= 8:
            raise ValueError(f"invalid launch shape ({b}, {c})")
        results[f"{b}x{c}"] = float(timer(b, c))
    if not results:
        raise ValueError("no launch shape to try")
    best = min(results, key=results.get)
    b, c = (int(x) for x in best.split("x"))
    _store(path, key, {"batch": b, "ctas_per_sm": c, "ms": results})
    return b, c


def config_for(scene, cams, base: Optional[abi.unigs_config] = None,
               cache_path: Optional[str] = None, tune_if_missing: bool = False):
    """A ``unigs_config`` with the cached launch shape for this workload (the
    library default when none is cached and ``tune_if_missing`` is false)."""
    path = cache_path or default_cache_path()
    hit = _load(path).get(workload_key(scene, cams))
    if hit:
        return make_config(hit["batch"], hit["ctas_per_sm"], base)
    if tune_if_missing:
        b, c = tune(scene, cams, base=base, cache_path=path)
        return make_config(b, c, base)
    return make_config(0, 0, base)
