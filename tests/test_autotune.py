"""Host logic of the launch-shape autotuner (no GPU): cache keys, the search
and the JSON cache; and, on a GPU, one real search on a small scene."""
import json

import pytest

from paper_2510_12174_gb300 import autotune


def test_key_classes():
    k = autotune.key_for("GB300", 152, 64, "bf16", [(1280, 720)] * 16, 1_000_000)
    assert k == "GB300|sm152|sem64|bf16|cams16|px2^24|n2^20"
    # logit counts share the kernel's compiled width
    assert autotune.key_for("G", 1, 5, "f32", [(8, 8)], 10).split("|")[2] == "sem8"
    assert autotune.key_for("G", 1, 17, "f32", [(8, 8)], 10).split("|")[2] == "sem32"
    assert autotune.key_for("G", 1, 0, "f32", [(8, 8)], 10).split("|")[2] == "sem0"
    assert autotune.key_for("G", 1, 100, "f32", [(8, 8)], 10).split("|")[2] == "sem64"


def test_search_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "shapes.json")
    cost = {(32, 2): 5.0, (16, 2): 4.0, (64, 1): 6.0}
    calls = []

    def timer(b, c):
        calls.append((b, c))
        return cost[(b, c)]

    assert autotune.search("k", "bwd", cost, path, False, timer) == (16, 2)
    assert len(calls) == 3
    d = json.load(open(path))
    assert d["k"]["bwd"]["batch"] == 16 and d["k"]["bwd"]["ms"]["64x1"] == 6.0
    # a cached key is not timed again unless forced
    assert autotune.search("k", "bwd", cost, path, False, timer) == (16, 2)
    assert len(calls) == 3
    cost[(64, 1)] = 1.0
    assert autotune.search("k", "bwd", cost, path, True, timer) == (64, 1)
    # the other stage and other keys are kept
    autotune.search("k", "fwd", {(16, 4): 1.0}, path, False, lambda b, c: 1.0)
    autotune.search("other", "bwd", {(32, 1): 1.0}, path, False, lambda b, c: 1.0)
    d = json.load(open(path))
    assert set(d) == {"k", "other"} and set(d["k"]) == {"fwd", "bwd"}
    assert d["k"]["bwd"]["batch"] == 64


def test_search_rejects_invalid_shapes(tmp_path):
    with pytest.raises(ValueError):
        autotune.search("k", "fwd", [(48, 2)], str(tmp_path / "s.json"), False,
                        lambda b, c: 1.0)
    with pytest.raises(ValueError):
        autotune.search("k", "fwd", [(32, 0)], str(tmp_path / "s.json"), False,
                        lambda b, c: 1.0)


def test_tile_search_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "shapes.json")
    cost = {(16, 16): 5.0, (32, 8): 4.0, (8, 32): 6.0, (64, 4): 4.5}
    calls = []

    def timer(tile):
        calls.append(tile)
        return cost[tile]

    assert autotune.search_tile("k", cost, path, False, timer) == (32, 8)
    assert len(calls) == 4
    assert autotune.search_tile("k", cost, path, False, timer) == (32, 8)
    assert len(calls) == 4
    d = json.load(open(path))
    assert d["k"]["tile"] == {"w": 32, "h": 8, "ms": {"16x16": 5.0, "32x8": 4.0, "8x32": 6.0,
                                                      "64x4": 4.5}}
    with pytest.raises(ValueError):
        autotune.search_tile("k2", [(16, 8)], path, False, timer)


def test_tune_chooses_tile_then_launch_shapes(tmp_path):
    path = str(tmp_path / "shapes.json")
    seen = []

    def tile_timer(tile):
        return {(16, 16): 3.0, (32, 8): 2.0}[tile]

    def timer(stage, b, c):
        seen.append((stage, b, c))
        return float(b * c)

    import paper_2510_12174_gb300.autotune as at
    key = at.key_for("G", 1, 16, "bf16", [(64, 48)], 4000)
    # workload_key needs a device: exercise the same steps with the key
    tile = at.search_tile(key, [(16, 16), (32, 8)], path, False, tile_timer)
    fwd = at.search(key, "fwd", [(16, 4), (32, 2)], path, False, lambda b, c: timer("fwd", b, c))
    bwd = at.search(key, "bwd", [(8, 3), (16, 1)], path, False, lambda b, c: timer("bwd", b, c))
    assert tile == (32, 8) and fwd == (16, 4) and bwd == (16, 1)
    d = json.load(open(path))[key]
    assert set(d) == {"tile", "fwd", "bwd"}


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "s.json"
    path.write_text("{not json")
    assert autotune.search("k", "bwd", [(32, 2)], str(path), False, lambda b, c: 1.0) == (32, 2)


@pytest.mark.gpu
def test_tune_on_small_scene(tmp_path):
    import torch
    import __graft_entry__ as ge
    from paper_2510_12174_gb300 import rasterizer as rz
    from paper_2510_12174_gb300 import scenes
    ge.build()
    sc, cams = scenes.small_room(n=4000, width=64, height=48, n_sem=16, seed=3, n_cams=2)
    ds = rz.DeviceScene.from_scene(sc)
    path = str(tmp_path / "s.json")
    best = autotune.tune(ds, cams, fwd_candidates=[(16, 4), (32, 2)],
                         bwd_candidates=[(32, 2), (16, 1)], reps=2, cache_path=path,
                         tile_candidates=[(16, 16), (32, 8)])
    assert best["tile"] in [(16, 16), (32, 8)]
    assert best["fwd"] in [(16, 4), (32, 2)] and best["bwd"] in [(32, 2), (16, 1)]
    cfg = autotune.config_for(ds, cams, cache_path=path)
    assert (cfg.batch, cfg.ctas_per_sm) == best["bwd"]
    assert (cfg.batch_fwd, cfg.ctas_per_sm_fwd) == best["fwd"]
    assert (cfg.tile_w, cfg.tile_h) == best["tile"]
    torch.cuda.synchronize()
