"""Parity on the named workload configurations (the benchmark's neighbours):

* config 1 - forward only, FP32, 10k Gaussians, one 256x256 camera: every pixel;
* config 2 - forward + backward, FP32, 200k room Gaussians, 640x480, 32 logits:
  binning bit-exact, forward and gradients on a two-row band of tiles;
* config 4 - batched, BF16 storage (tensor-core logit blend), 3M Gaussians,
  16 orbit cameras of mixed resolution: per-camera binning bit-exact for one
  camera of each resolution and sampled pixels against the oracle;
* config 5 - the training loss at full size (8 views at 1920x1080, 64
  logits) on seeded stand-in maps: every sum and weight, sampled gradients.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import raster as orr
from oracle import train as ot
from paper_2510_12174_gb300 import abi
from paper_2510_12174_gb300 import rasterizer as rz
from paper_2510_12174_gb300 import scenes

from gpu_helpers import (MAX_AMBIGUOUS_FWD, MAX_AMBIGUOUS_GRAD, TOL_ABS, TOL_REL,
                         check_grad_errors, flat_upstream, forward_errors, grad_errors,
                         masked_upstream, sampled_errors)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    torch.cuda.set_device(0)


def _render(sc, cams, **kw):
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams, **kw)
    out = r.forward()
    torch.cuda.synchronize()
    return r, out


def test_config1_forward_every_pixel():
    sc, cams = scenes.config1()
    r, out = _render(sc, cams)
    keys, vals, ranges = r.sorted_instances()
    ref_b = oracle.bin_cameras_fast(sc, cams)
    assert np.array_equal(keys, ref_b["keys"]) and np.array_equal(vals, ref_b["vals"])
    assert np.array_equal(ranges, ref_b["ranges"])
    _, ref, _ = oracle.render(sc, cams, binning=ref_b, with_normal_d=False)
    e = forward_errors(r, out, ref, sc.n_sem)
    print("config1", e)
    assert e["ambiguous_fraction"] < MAX_AMBIGUOUS_FWD and e["n_contrib"] == 0
    assert e["rgb"] < TOL_ABS and e["normal_g"] < TOL_ABS and e["kmap"] < TOL_ABS
    assert e["T_final"] < TOL_ABS
    assert e["depth"] < TOL_REL and e["logits"] < TOL_REL


def _band_errors(r, out, ref, band_mask, n_sem):
    """Max forward errors over the band's non-ambiguous pixels."""
    ok = band_mask & ~ref["amb_fwd"].numpy()
    got = {k: r.split(out[k], c)[0].cpu().numpy() for k, c in
           (("rgb", 3), ("depth", 1), ("normal_g", 3), ("kmap", 1), ("T_final", 1),
            ("logits", n_sem))}
    e = {}
    for k, rk in (("rgb", "rgb"), ("normal_g", "normal"), ("kmap", "kmap"), ("T_final", "T")):
        g, x = got[k], ref[rk].numpy()
        e[k] = float(np.abs(g - x)[..., ok].max())
    for k, rk in (("depth", "depth"), ("logits", "logits")):
        g, x = got[k], ref[rk].numpy()
        rms = np.sqrt(np.mean(x[..., ok] ** 2))
        e[k] = float((np.abs(g - x) / np.maximum(np.abs(x), rms))[..., ok].max())
    return e, int(band_mask.sum() - ok.sum())


def test_config2_band_forward_and_gradients():
    sc, cams = scenes.config2()
    cam = cams[0]
    r, out = _render(sc, cams)
    ref_b = oracle.bin_cameras_fast(sc, cams)
    keys, vals, ranges = r.sorted_instances()
    assert np.array_equal(keys, ref_b["keys"]) and np.array_equal(vals, ref_b["vals"])
    assert np.array_equal(ranges, ref_b["ranges"])
    TX = (cam.width + 15) // 16
    band = list(range(12 * TX, 14 * TX))          # tile rows 12 and 13
    mask = np.zeros((cam.height, cam.width), dtype=bool)
    mask[12 * 16:14 * 16, :] = True
    _, ref, _ = oracle.render(sc, cams, binning=ref_b, tiles=[band], with_normal_d=False)
    e, n_amb = _band_errors(r, out, ref[0], mask, sc.n_sem)
    print("config2 band", e, "ambiguous", n_amb)
    assert n_amb < MAX_AMBIGUOUS_FWD * mask.sum()
    assert e["rgb"] < TOL_ABS and e["normal_g"] < TOL_ABS and e["kmap"] < TOL_ABS
    assert e["T_final"] < TOL_ABS and e["depth"] < TOL_REL and e["logits"] < TOL_REL
    # gradients of a loss on the band only
    up = scenes.upstream_grads(cams, sc.n_sem, seed=41)
    assert ref[0]["amb_grad"].numpy()[mask].mean() < MAX_AMBIGUOUS_GRAD
    drop = ~mask | ref[0]["amb_grad"].numpy()
    up = masked_upstream(up, [drop])
    up["normal_d"] = [np.zeros_like(x) for x in up["normal_d"]]
    _, gref, _ = oracle.render_and_grad(sc, cams, up, binning=ref_b, tiles=[band])
    fu = flat_upstream(up)
    grads = r.backward(out, {k: fu[k] for k in fu if k != "normal_d"})
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    check_grad_errors(grad_errors(grads, gref))


def test_config4_batched_mixed_resolution():
    sc, cams = scenes.config4()
    r, out = _render(sc, cams)
    assert r.status()[0] == 0
    keys, vals, ranges = r.sorted_instances()
    tile_off = [int(r.plan.tile_offset[k]) for k in range(len(cams) + 1)]
    seen = {}
    for k, c in enumerate(cams):
        seen.setdefault((c.width, c.height), k)
    rng = np.random.default_rng(5)
    for (w, h), k in sorted(seen.items()):
        cam = cams[k]
        ref_b = oracle.bin_cameras_fast(sc, [cam])
        t0, t1 = tile_off[k], tile_off[k + 1]
        rk = ranges[t0:t1]
        s0, s1 = int(rk[rk[:, 1] > rk[:, 0]][:, 0].min()), int(rk[:, 1].max())
        k_loc = keys[s0:s1] - (np.uint64(t0) << np.uint64(32))
        assert np.array_equal(k_loc, ref_b["keys"]), (w, h)
        assert np.array_equal(vals[s0:s1], ref_b["vals"]), (w, h)
        loc = rk.astype(np.int64) - s0
        loc[rk[:, 1] == rk[:, 0]] = 0
        refr = ref_b["ranges"].astype(np.int64)
        refr[ref_b["ranges"][:, 1] == ref_b["ranges"][:, 0]] = 0
        assert np.array_equal(loc, refr), (w, h)
        # sampled pixels against the oracle
        params = orr.Params.from_scene(sc)
        with torch.no_grad():
            prep = orr.preprocess(params, cam)
        TX = (cam.width + 15) // 16
        views = {key: r.split(out[key], ch)[k].cpu().numpy() for key, ch in
                 (("rgb", 3), ("depth", 1), ("normal_g", 3), ("kmap", 1), ("logits", 64))}
        okey = {"rgb": "rgb", "depth": "depth", "normal_g": "normal", "kmap": "kmap",
                "logits": "logits"}
        got = {key: [] for key in views}
        exp = {key: [] for key in views}
        n_amb = 0
        for _ in range(40):
            u, v = int(rng.integers(0, cam.width)), int(rng.integers(0, cam.height))
            t = (v // 16) * TX + (u // 16)
            a0, a1 = ref_b["ranges"][t]
            ids = torch.as_tensor(ref_b["vals"][a0:a1].astype(np.int64))
            with torch.no_grad():
                rr = orr.composite_tile(prep, ids, torch.tensor([[float(u), float(v)]],
                                                                dtype=torch.float64), cam)
            if bool(rr["amb_fwd"][0]):
                n_amb += 1
                continue
            for key in views:
                got[key].append(np.atleast_1d(views[key][..., v, u]))
                exp[key].append(np.atleast_1d(rr[okey[key]][0].numpy()))
        worst = sampled_errors(got, exp)
        print("config4", (w, h), worst, "ambiguous", n_amb)
        assert n_amb <= 2
        assert worst["rgb"] < TOL_ABS and worst["normal_g"] < TOL_ABS
        assert worst["kmap"] < TOL_ABS and worst["depth"] < TOL_REL
        assert worst["logits"] < TOL_REL


def test_config5_loss_at_full_size():
    """8 views at 1920x1080, 64 logits: the loss kernels on seeded stand-in
    maps against the oracle, which takes the terms per camera (float64) and
    pools their sums."""
    cams = scenes.orbit_cameras(8, seed=15, resolutions=[(1920, 1080)])
    n_sem = 64
    maps = scenes.synthetic_maps(cams, n_sem, seed=51)
    tgt = scenes.synthetic_targets(cams, n_sem, seed=52)
    sc, _ = scenes.small_room(n=50, n_sem=n_sem, seed=30)
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams)
    dev = {k: torch.as_tensor(np.concatenate([a.ravel() for a in v]), device="cuda")
           for k, v in maps.items()}
    out = {"rgb": dev["rgb"], "depth": dev["depth"], "kmap": dev["kmap"],
           "logits": dev["logits"], "normal_d": dev["normal_d"],
           "normal_g": None, "T_final": None, "n_contrib": None}
    dtg = {k: torch.as_tensor(np.concatenate([a.ravel() for a in v]), device="cuda")
           for k, v in tgt.items()}
    record = torch.zeros(16, device="cuda")
    lg = r.alloc_loss_grads()
    r.loss(out, dtg, record, lg)
    torch.cuda.synchronize()
    rec = record.cpu().numpy()
    # oracle: terms per camera, pooled
    sums = {"l1": 0.0, "normal": 0.0, "depth": 0.0, "seg": 0.0, "K": 0.0}
    n_d = n_l = 0
    P = 0
    per_cam = []
    for k in range(len(cams)):
        m = {key: [np.asarray(maps[key][k], dtype=np.float64)] for key in maps}
        t = {key: [tgt[key][k]] for key in tgt}
        terms = ot.loss_terms(m, t)
        Pk = cams[k].width * cams[k].height
        nd = int((tgt["depth"][k] > 0).sum())
        lab = tgt["label"][k]
        nl = int(((lab >= 0) & (lab < n_sem)).sum())
        sums["l1"] += terms["l1"][0] * 3 * Pk
        sums["normal"] += (1.0 - terms["normal"][0]) * Pk
        sums["depth"] += terms["depth"][0] * nd
        sums["seg"] += terms["seg"][0] * nl
        sums["K"] += terms["K"][0] * Pk
        n_d, n_l, P = n_d + nd, n_l + nl, P + Pk
        per_cam.append(terms)
    L = {"l1": sums["l1"] / (3 * P), "normal": 1.0 - sums["normal"] / P,
         "depth": sums["depth"] / n_d, "seg": sums["seg"] / n_l, "K": sums["K"] / P}
    total, w, _ = ot.combine({k: (v, {}) for k, v in L.items()})
    for i, k in enumerate(("l1", "normal", "depth", "seg", "K")):
        assert rec[1 + i] == pytest.approx(L[k], rel=1e-5), k
        assert rec[6 + i] == pytest.approx(w[k], rel=1e-5), k
    assert rec[0] == pytest.approx(total, rel=1e-5)
    assert rec[abi.UNIGS_LOSS_N_DEPTH] == n_d and rec[abi.UNIGS_LOSS_N_LABEL] == n_l
    # gradients at sampled pixels: the per-camera oracle gradient rescaled
    # from that camera's normalisation to the pooled one
    g = {k: v.cpu().numpy() for k, v in lg.items()}
    offs = r.pixel_offsets()
    rng = np.random.default_rng(53)
    for k in rng.choice(len(cams), 3, replace=False):
        terms = per_cam[k]
        Pk = cams[k].width * cams[k].height
        nd = int((tgt["depth"][k] > 0).sum())
        lab = tgt["label"][k]
        nl = int(((lab >= 0) & (lab < n_sem)).sum())
        scale = {"rgb": w["l1"] * (3 * Pk) / (3 * P), "normal_d": w["normal"] * Pk / P,
                 "depth": w["depth"] * nd / n_d, "logits": w["seg"] * nl / n_l,
                 "kmap": w["K"] * Pk / P}
        src = {"rgb": ("l1", "rgb", 3), "normal_d": ("normal", "normal_d", 3),
               "depth": ("depth", "depth", 1), "logits": ("seg", "logits", n_sem),
               "kmap": ("K", "kmap", 1)}
        idx = rng.integers(0, Pk, 2000)
        for key, (term, gk, ch) in src.items():
            ref = np.asarray(terms[term][1][gk][0]).reshape(ch, Pk)[:, idx] * scale[key]
            got = g[key][offs[k] * ch: offs[k + 1] * ch].reshape(ch, Pk)[:, idx]
            err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30)
            assert err < 1e-5, (key, err)
