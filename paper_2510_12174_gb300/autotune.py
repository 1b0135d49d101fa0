"""Tile-shape and launch-shape autotuner of the composite kernels.

The composites (forward Alg. 2 and backward Alg. 4) are persistent kernels
whose CTAs pull tiles of 256 pixels from a device work counter, longest
Gaussian list first.  The tile shape (16 x 16, 8 x 32, 32 x 8 or 64 x 4)
decides how many (tile, Gaussian) pairs the binning lists and how well a tile's
pixels share its Gaussians; it does not change the image (each Gaussian is
drawn on the pixels of its 3-sigma square, whatever tiles list it).  Two launch
parameters per kernel change their speed but not their results:

* the batch: Gaussians staged per shared-memory batch (8 - backward only -,
  16, 32 or 64).  Larger
  batches amortise the barrier and bulk-copy issue per Gaussian; smaller ones
  waste less of the last batch of short lists and need less shared memory.
* CTAs per SM (1-4): more CTAs hide barrier, MMA and atomic latency; fewer
  leave more registers and shared memory per CTA.

The forward output is bit-identical for every shape on the FP32-pipe path
(each pixel blends its list in the same order) and moves by float32 summation
order on the tensor-core logit blend; the gradients move by the order of
float32 atomic additions.

:func:`tune` first times one forward + backward step per tile shape at the
library's default launch shapes and keeps the fastest shape; at that shape it
times the forward candidates on the forward alone and the backward candidates
on the backward alone (CUDA events on the caller's scene and cameras), keeps
the fastest of each, and caches all three in a JSON file keyed
by :func:`workload_key` (GPU, SM count, logit class, feature dtype, camera
count and pixel/Gaussian magnitudes), so a training run pays the search once
per workload class.  :func:`config_for` returns a ``unigs_config`` with the
cached tile and launch shapes (or the library defaults).
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, Optional, Sequence, Tuple

import torch

from . import abi
from . import rasterizer as rz

TILE_CANDIDATES: Tuple[Tuple[int, int], ...] = tuple(abi.TILE_SHAPES)
FWD_CANDIDATES: Tuple[Tuple[int, int], ...] = ((16, 4), (16, 3), (32, 2), (16, 2), (64, 2))
BWD_CANDIDATES: Tuple[Tuple[int, int], ...] = ((8, 3), (32, 2), (16, 2), (8, 2), (64, 1))


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


def make_config(batch: int = 0, ctas_per_sm: int = 0, base: Optional[abi.unigs_config] = None,
                batch_fwd: int = 0, ctas_per_sm_fwd: int = 0, tile=None):
    cfg = (abi.unigs_config.from_buffer_copy(base) if base is not None
           else abi.unigs_config_default())
    cfg.batch, cfg.ctas_per_sm = int(batch), int(ctas_per_sm)
    cfg.batch_fwd, cfg.ctas_per_sm_fwd = int(batch_fwd), int(ctas_per_sm_fwd)
    if tile is not None:
        cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
    return cfg


def _synthetic_upstream(r: "rz.Renderer", seed: int) -> Dict[str, torch.Tensor]:
    g = torch.Generator(device=r.device).manual_seed(seed)
    P = r.n_pixels
    f = lambda c: torch.randn(c * P, generator=g, device=r.device)
    up = {"rgb": f(3), "depth": f(1), "normal_g": f(3), "kmap": f(1)}
    up["logits"] = f(r.scene.n_sem) if r.scene.n_sem else None
    return up


def _median_ms(fn, stream, reps: int) -> float:
    times = []
    for _ in range(max(1, reps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def time_tile(scene, cams, tile, reps: int = 3, base: Optional[abi.unigs_config] = None,
              seed: int = 0) -> float:
    """Milliseconds of one forward + backward step (preprocess, binning,
    forward composite, backward) at the tile shape and the default launch
    shapes, median of ``reps`` after one warm-up."""
    r = rz.Renderer(scene, cams, cfg=make_config(0, 0, base, 0, 0, tile))
    out = r.forward()                       # sizes the instance capacity
    stream = torch.cuda.current_stream(r.device)
    up = _synthetic_upstream(r, seed)
    grads = r.alloc_grads()

    def step():
        r.forward(out, readback=False, normal_d=False)
        r.backward(out, up, grads=grads)

    step()
    ms = _median_ms(step, stream, reps)
    s, _ = r.status()
    abi.check(s, f"tile shape {tile}")
    return ms


def time_shape(scene, cams, batch: int, ctas_per_sm: int, reps: int = 3,
               base: Optional[abi.unigs_config] = None, seed: int = 0,
               stage: str = "bwd", tile=None) -> float:
    """Milliseconds of the forward composite (stage "fwd": preprocess, sort
    and forward at the shape) or of the backward (stage "bwd"), median of
    ``reps`` after one warm-up."""
    cfg = (make_config(0, 0, base, batch, ctas_per_sm, tile) if stage == "fwd"
           else make_config(batch, ctas_per_sm, base, tile=tile))
    r = rz.Renderer(scene, cams, cfg=cfg)
    out = r.forward()                       # sizes the instance capacity
    stream = torch.cuda.current_stream(r.device)
    if stage == "fwd":
        ms = _median_ms(lambda: r.forward(out, readback=False, normal_d=False), stream, reps)
    else:
        up = _synthetic_upstream(r, seed)
        grads = r.alloc_grads()
        r.backward(out, up, grads=grads)
        ms = _median_ms(lambda: r.backward(out, up, grads=grads), stream, reps)
    s, _ = r.status()
    abi.check(s, f"launch shape ({batch}, {ctas_per_sm})")
    return ms


def tune(scene, cams, fwd_candidates: Iterable[Tuple[int, int]] = FWD_CANDIDATES,
         bwd_candidates: Iterable[Tuple[int, int]] = BWD_CANDIDATES, reps: int = 3,
         base: Optional[abi.unigs_config] = None, cache_path: Optional[str] = None,
         force: bool = False, timer=None,
         tile_candidates: Iterable[Tuple[int, int]] = TILE_CANDIDATES,
         tile_timer=None) -> Dict[str, Tuple[int, int]]:
    """Fastest tile shape, then the fastest forward and backward (batch,
    ctas_per_sm) at that tile, for this scene and camera set, cached:
    {"tile": (w, h), "fwd": (b, c), "bwd": (b, c)}.

    ``tile_timer(tile) -> ms`` and ``timer(stage, batch, ctas_per_sm) -> ms``
    replace the CUDA-event timings of :func:`time_tile` and
    :func:`time_shape`."""
    path = cache_path or default_cache_path()
    key = workload_key(scene, cams)
    tt = tile_timer or (lambda tl: time_tile(scene, cams, tl, reps=reps, base=base))
    tile = search_tile(key, tile_candidates, path, force, tt)
    t = timer or (lambda st, b, c: time_shape(scene, cams, b, c, reps=reps, base=base, stage=st,
                                              tile=tile))
    return {"tile": tile,
            "fwd": search(key, "fwd", fwd_candidates, path, force, lambda b, c: t("fwd", b, c)),
            "bwd": search(key, "bwd", bwd_candidates, path, force, lambda b, c: t("bwd", b, c))}


def search_tile(key: str, candidates: Iterable[Tuple[int, int]], path: str, force: bool,
                timer) -> Tuple[int, int]:
    """Cache lookup of the tile shape of ``key``, else time every candidate
    and store the fastest."""
    if not force:
        hit = _load(path).get(key, {}).get("tile")
        if hit:
            return int(hit["w"]), int(hit["h"])
    results = {}
    for w, h in candidates:
        if (int(w), int(h)) not in abi.TILE_SHAPES:
            raise ValueError(f"invalid tile shape ({w}, {h})")
        results[f"{w}x{h}"] = float(timer((int(w), int(h))))
    if not results:
        raise ValueError("no tile shape to try")
    best = min(results, key=results.get)
    w, h = (int(x) for x in best.split("x"))
    entry = _load(path).get(key, {})
    entry["tile"] = {"w": w, "h": h, "ms": results}
    _store(path, key, entry)
    return w, h


def search(key: str, slot: str, candidates: Iterable[Tuple[int, int]], path: str, force: bool,
           timer) -> Tuple[int, int]:
    """Cache lookup of ``key``/``slot``, else time every candidate and store
    the fastest."""
    if not force:
        hit = _load(path).get(key, {}).get(slot)
        if hit:
            return int(hit["batch"]), int(hit["ctas_per_sm"])
    results = {}
    for b, c in candidates:
        if b not in ((8, 16, 32, 64) if slot == "bwd" else (16, 32, 64)) or not 1 <= c <= 8:
            raise ValueError(f"invalid launch shape ({b}, {c})")
        results[f"{b}x{c}"] = float(timer(b, c))
    if not results:
        raise ValueError("no launch shape to try")
    best = min(results, key=results.get)
    b, c = (int(x) for x in best.split("x"))
    entry = _load(path).get(key, {})
    entry[slot] = {"batch": b, "ctas_per_sm": c, "ms": results}
    _store(path, key, entry)
    return b, c


def config_for(scene, cams, base: Optional[abi.unigs_config] = None,
               cache_path: Optional[str] = None, tune_if_missing: bool = False):
    """A ``unigs_config`` with the cached launch shapes for this workload (the
    library defaults for a stage without an entry, unless
    ``tune_if_missing``)."""
    path = cache_path or default_cache_path()
    hit = _load(path).get(workload_key(scene, cams), {})
    if tune_if_missing and not ("fwd" in hit and "bwd" in hit and "tile" in hit):
        tune(scene, cams, base=base, cache_path=path)
        hit = _load(path).get(workload_key(scene, cams), {})
    f, b, tl = hit.get("fwd", {}), hit.get("bwd", {}), hit.get("tile")
    return make_config(b.get("batch", 0), b.get("ctas_per_sm", 0), base,
                       f.get("batch", 0), f.get("ctas_per_sm", 0),
                       (tl["w"], tl["h"]) if tl else None)


def main(argv=None):
    """Tunes the launch shapes of the synthetic-room workload of the benchmark
    (or a smaller one) and prints the measured candidates as JSON."""
    import argparse

    from . import scenes
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--gaussians", type=int, default=1_000_000)
    ap.add_argument("--views", type=int, default=16)
    ap.add_argument("--fp32", action="store_true", help="float32 feature storage")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cache", default=None, help="cache file (default: the user cache)")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    sc, cams = scenes.config3_orbit(args.views, n=args.gaussians, feat_bf16=not args.fp32)
    ds = rz.DeviceScene.from_scene(sc)
    path = args.cache or default_cache_path()
    best = tune(ds, cams, reps=args.reps, cache_path=path, force=True)
    entry = _load(path).get(workload_key(ds, cams), {})
    print(json.dumps({"workload": workload_key(ds, cams), "best": best,
                      "tile_ms": entry.get("tile", {}).get("ms"),
                      "fwd_ms": entry.get("fwd", {}).get("ms"),
                      "bwd_ms": entry.get("bwd", {}).get("ms")}, indent=1))


if __name__ == "__main__":
    main()
