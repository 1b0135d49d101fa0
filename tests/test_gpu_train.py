"""GPU parity of the training step (include/unigs_train.h) against the FP64
oracle in oracle/train.py: the combined loss and its gradients, Adam with
activations and bfloat16 copies, the pruning compaction; and the Trainer
(loss decreases, prune, checkpoint round trip)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import train as ot
from paper_2510_12174_gb300 import abi
from paper_2510_12174_gb300 import rasterizer as rz
from paper_2510_12174_gb300 import scenes
from paper_2510_12174_gb300 import train as tr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    torch.cuda.set_device(0)


def _flat(maps, dtype=torch.float32):
    return torch.as_tensor(np.concatenate([np.asarray(a).ravel() for a in maps]),
                           dtype=dtype, device="cuda")


def _split(flat, cams, channels):
    res, a = [], 0
    for c in cams:
        n = channels * c.width * c.height
        x = flat[a:a + n].reshape((channels, c.height, c.width) if channels > 1
                                  else (c.height, c.width))
        res.append(x)
        a += n
    return res


def _run_loss(cams, n_sem, maps, tgt, drop=()):
    sc, _ = scenes.small_room(n=50, n_sem=n_sem, seed=30)
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams)
    dev = {k: _flat(v) for k, v in maps.items()}
    out = abi.unigs_outputs()
    out.rgb, out.depth, out.kmap = dev["rgb"].data_ptr(), dev["depth"].data_ptr(), dev["kmap"].data_ptr()
    out.logits = dev["logits"].data_ptr() if n_sem else None
    t = abi.unigs_targets()
    td = {"rgb": _flat(tgt["rgb"]), "depth": _flat(tgt["depth"]), "normal": _flat(tgt["normal"]),
          "label": _flat(tgt["label"], torch.int32)}
    for k in ("rgb", "depth", "normal", "label"):
        setattr(t, k, None if k in drop else td[k].data_ptr())
    lam = abi.unigs_loss_lambda()
    abi.lib().unigs_loss_lambda_default(ctypes.byref(lam))
    P = r.n_pixels
    g = {k: torch.full((c * P,), 7.0, device="cuda") for k, c in
         (("rgb", 3), ("depth", 1), ("normal_d", 3), ("kmap", 1), ("logits", n_sem))}
    gs = abi.unigs_loss_grads()
    for k, v in g.items():
        setattr(gs, k, v.data_ptr() if v.numel() else None)
    rec = torch.full((abi.UNIGS_LOSS_RECORD_FLOATS,), -1.0, device="cuda")
    abi.check(abi.lib().unigs_loss(ctypes.byref(r.plan), ctypes.byref(out),
                                   dev["normal_d"].data_ptr(), ctypes.byref(t),
                                   ctypes.byref(lam), r.ws.data_ptr(), rec.data_ptr(),
                                   ctypes.byref(gs), r._stream()), "unigs_loss")
    torch.cuda.synchronize()
    return rec.cpu().numpy(), {k: v.cpu().numpy() for k, v in g.items()}


def _oracle_loss(maps, tgt):
    m64 = {k: [np.asarray(a, dtype=np.float64) for a in v] for k, v in maps.items()}
    terms = ot.loss_terms(m64, tgt)
    return terms, ot.combine(terms)


@pytest.mark.parametrize("n_sem", [8, 64])
def test_loss_values_and_gradients(n_sem):
    _, cams = scenes.small_room(n=50, n_sem=n_sem, seed=30, n_cams=2, width=61, height=45)
    maps = scenes.synthetic_maps(cams, n_sem, seed=31)
    tgt = scenes.synthetic_targets(cams, n_sem, seed=32)
    rec, g = _run_loss(cams, n_sem, maps, tgt)
    terms, (total, w, grads) = _oracle_loss(maps, tgt)
    idx = {"l1": 1, "normal": 2, "depth": 3, "seg": 4, "K": 5}
    for k, i in idx.items():
        assert rec[i] == pytest.approx(terms[k][0], rel=1e-5), k
        assert rec[5 + i] == pytest.approx(w[k], rel=1e-5), k
    assert rec[0] == pytest.approx(total, rel=1e-5)
    for key, ch in (("rgb", 3), ("depth", 1), ("normal_d", 3), ("kmap", 1), ("logits", n_sem)):
        ref = np.concatenate([a.ravel() for a in grads[key]])
        scale = np.abs(ref).max()
        err = np.abs(g[key] - ref).max() / scale
        assert err < 1e-5, (key, err)
        # sign decisions of the L1 subgradients are exact
        if key in ("rgb", "depth", "kmap"):
            assert np.array_equal(np.sign(g[key]), np.sign(ref)), key


def test_loss_degenerate_targets():
    """No depth measurement and every pixel unlabelled: those terms, weights
    and gradients are 0; dropped targets write zero gradients."""
    _, cams = scenes.small_room(n=50, n_sem=8, seed=30, n_cams=1, width=40, height=33)
    maps = scenes.synthetic_maps(cams, 8, seed=33)
    tgt = scenes.synthetic_targets(cams, 8, seed=34)
    tgt["depth"] = [np.zeros_like(a) for a in tgt["depth"]]
    tgt["label"] = [np.full_like(a, -1) for a in tgt["label"]]
    tgt["label"][0][0, 0] = 8           # out of range: unlabelled too
    rec, g = _run_loss(cams, 8, maps, tgt)
    assert rec[abi.UNIGS_LOSS_DEPTH] == 0 and rec[abi.UNIGS_LOSS_W_DEPTH] == 0
    assert rec[abi.UNIGS_LOSS_SEG] == 0 and rec[abi.UNIGS_LOSS_N_LABEL] == 0
    assert np.all(g["depth"] == 0) and np.all(g["logits"] == 0)
    terms, (total, _, _) = _oracle_loss(maps, tgt)
    assert rec[0] == pytest.approx(total, rel=1e-5)
    rec2, g2 = _run_loss(cams, 8, maps, tgt, drop=("rgb", "normal"))
    assert rec2[abi.UNIGS_LOSS_L1] == 0 and np.all(g2["rgb"] == 0)
    assert np.all(g2["normal_d"] == 0)
    # with L_l1 = 0 every normalised weight is 0 as well
    assert rec2[0] == 0 and np.all(g2["kmap"] == 0)


def _adam_groups(arrs, acts, lrs, with_copies=True):
    groups = (abi.unigs_adam_group * len(arrs))()
    for i, (a, act, lr) in enumerate(zip(arrs, acts, lrs)):
        G = groups[i]
        G.param, G.grad, G.m, G.v = (a["raw"].data_ptr(), a["g"].data_ptr(), a["m"].data_ptr(),
                                     a["v"].data_ptr())
        if with_copies:
            G.act_out, G.bf16_out = a["act"].data_ptr(), a["b16"].data_ptr()
        G.count, G.lr, G.activation = a["raw"].numel(), lr, act
    return groups


def test_adam_matches_oracle_over_steps():
    rng = np.random.default_rng(40)
    acts = [abi.UNIGS_ACT_NONE, abi.UNIGS_ACT_EXP, abi.UNIGS_ACT_SIGMOID]
    lrs = [1e-2, 5e-3, 5e-2]
    sizes = [10001, 3 * 777, 1]
    host = []
    dev = []
    for n in sizes:
        raw = rng.normal(0, 1, n).astype(np.float32)
        host.append({"raw": raw.astype(np.float64), "m": np.zeros(n), "v": np.zeros(n)})
        dev.append({"raw": torch.tensor(raw, device="cuda"),
                    "m": torch.zeros(n, device="cuda"), "v": torch.zeros(n, device="cuda"),
                    "act": torch.zeros(n, device="cuda"),
                    "b16": torch.zeros(n, dtype=torch.bfloat16, device="cuda"),
                    "g": torch.zeros(n, device="cuda")})
    hp = abi.unigs_adam_hparams(0.9, 0.999, 1e-8)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for t in range(1, 4):
        for h, d in zip(host, dev):
            gg = rng.normal(0, 1, d["raw"].numel()).astype(np.float32)
            d["g"].copy_(torch.tensor(gg))
            h["g"] = gg.astype(np.float64)
        abi.check(abi.lib().unigs_adam_step(_adam_groups(dev, acts, lrs), 3, ctypes.byref(hp),
                                            step.data_ptr(), st), "unigs_adam_step")
        for h, act, lr in zip(host, acts, lrs):
            h["raw"], h["m"], h["v"], h["act"] = ot.adam_step(h["raw"], h["g"], h["m"], h["v"], t,
                                                              lr, 0.9, 0.999, 1e-8, act)
    torch.cuda.synchronize()
    assert int(step.item()) == 3
    for h, d in zip(host, dev):
        for k in ("raw", "m", "v", "act"):
            got = d[k].cpu().numpy().astype(np.float64)
            err = np.abs(got - h[k]).max() / max(np.abs(h[k]).max(), 1e-30)
            assert err < 2e-5, (k, err)
        # the bfloat16 copy is the round-to-nearest-even of the float32 copy
        b16 = d["b16"].float().cpu().numpy()
        assert np.array_equal(b16, scenes.round_to_bf16(d["act"].cpu().numpy()))


def test_param_copies_and_argument_checks():
    raw = torch.linspace(-3, 3, 999, device="cuda")
    act = torch.zeros_like(raw)
    b16 = torch.zeros(999, dtype=torch.bfloat16, device="cuda")
    groups = (abi.unigs_adam_group * 1)()
    G = groups[0]
    G.param, G.act_out, G.bf16_out, G.count, G.activation = (raw.data_ptr(), act.data_ptr(),
                                                             b16.data_ptr(), 999,
                                                             abi.UNIGS_ACT_SIGMOID)
    st = torch.cuda.current_stream().cuda_stream
    abi.check(abi.lib().unigs_param_copies(groups, 1, st))
    torch.cuda.synchronize()
    ref = 1 / (1 + np.exp(-raw.cpu().numpy().astype(np.float64)))
    assert np.abs(act.cpu().numpy() - ref).max() < 1e-6
    G.act_out = G.param  # an activated copy over the raw values
    assert abi.lib().unigs_param_copies(groups, 1, st) == abi.UNIGS_ERR_INVALID_ARG
    G.activation = 7
    assert abi.lib().unigs_param_copies(groups, 1, st) == abi.UNIGS_ERR_INVALID_ARG
    hp = abi.unigs_adam_hparams(0.9, 0.999, 1e-8)
    assert abi.lib().unigs_adam_step(groups, 17, ctypes.byref(hp), None, st) == \
        abi.UNIGS_ERR_INVALID_ARG


def test_prune_compaction_bit_exact():
    rng = np.random.default_rng(41)
    n = 50_003
    k = rng.uniform(0.6, 1.4, n).astype(np.float32)
    k[:4] = np.array([1.2, 0.8, 1.0 + np.float32(0.2), 1.0 - np.float32(0.2)], dtype=np.float32)
    keep = ot.prune_mask(k, 0.2)
    mean = rng.normal(size=(3, n)).astype(np.float32)
    sh = scenes.round_to_bf16(rng.normal(size=(n, 16, 3))).astype(np.float32)
    kd = torch.tensor(k, device="cuda")
    ws = torch.empty(abi.lib().unigs_prune_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    nk = ctypes.c_int64(0)
    st = torch.cuda.current_stream().cuda_stream
    abi.check(abi.lib().unigs_prune_mark(kd.data_ptr(), n, 0.2, ws.data_ptr(), ctypes.byref(nk), st))
    assert nk.value == int(keep.sum())
    md = torch.tensor(mean, device="cuda")
    shd = torch.tensor(sh, device="cuda").to(torch.bfloat16)
    m_out = torch.empty((3, nk.value), device="cuda")
    sh_out = torch.empty((nk.value, 16, 3), dtype=torch.bfloat16, device="cuda")
    k_out = torch.empty(nk.value, device="cuda")
    arr = (abi.unigs_prune_array * 3)()
    arr[0].src, arr[0].dst, arr[0].planes, arr[0].row, arr[0].elem_bytes = (
        md.data_ptr(), m_out.data_ptr(), 3, 1, 4)
    arr[1].src, arr[1].dst, arr[1].planes, arr[1].row, arr[1].elem_bytes = (
        shd.data_ptr(), sh_out.data_ptr(), 1, 48, 2)
    arr[2].src, arr[2].dst, arr[2].planes, arr[2].row, arr[2].elem_bytes = (
        kd.data_ptr(), k_out.data_ptr(), 1, 1, 4)
    arr[2].fill, arr[2].fill_value = 1, 0.9
    abi.check(abi.lib().unigs_prune_compact(arr, 3, n, nk.value, ws.data_ptr(), st))
    torch.cuda.synchronize()
    assert np.array_equal(m_out.cpu().numpy(), mean[:, keep])
    assert np.array_equal(sh_out.float().cpu().numpy(), sh[keep])
    assert np.all(k_out.cpu().numpy() == np.float32(0.9))
    # aliasing and bad element sizes are refused on the host
    arr[0].dst = arr[0].src
    assert abi.lib().unigs_prune_compact(arr, 3, n, nk.value, ws.data_ptr(), st) == \
        abi.UNIGS_ERR_INVALID_ARG


def _trainer_case(n=3000, seed=50):
    sc, cams = scenes.small_room(n=n, width=64, height=48, n_sem=8, seed=seed, n_cams=2)
    target_scene = scenes.perturb(sc, seed=seed + 1)
    _, ref, _ = oracle.render(target_scene, cams)
    tgt = {"rgb": _flat([r["rgb"].numpy() for r in ref]),
           "depth": _flat([r["depth"].numpy() for r in ref]),
           "normal": _flat([r["normal_d"].numpy() for r in ref]),
           "label": _flat([np.argmax(r["logits"].numpy(), axis=0) for r in ref], torch.int32)}
    return sc, cams, tgt


def test_trainer_loss_decreases_prunes_and_checkpoints(tmp_path):
    sc, cams, tgt = _trainer_case()
    cfg = tr.TrainConfig(prune_every=0)
    T = tr.Trainer.from_scene(sc, cams, tgt, cfg)
    T.step()
    first = T.losses()["total"]
    for _ in range(29):
        T.step()
    T.forward()
    T.loss()
    last = T.losses()["total"]
    assert np.isfinite(last) and last < 0.95 * first, (first, last)
    # prune: survivors in order, k reset to 0.9 and its moments to 0
    k_before = T.raw["k"].cpu().numpy()
    mean_before = T.raw["mean"].cpu().numpy()
    keep = ot.prune_mask(k_before, cfg.T_k)
    nk = T.prune()
    assert nk == int(keep.sum()) and T.n == nk and 0 < nk < len(k_before)
    assert np.array_equal(T.raw["mean"].cpu().numpy(), mean_before[:, keep])
    assert np.all(T.raw["k"].cpu().numpy() == np.float32(0.9))
    assert torch.all(T.m["k"] == 0) and torch.all(T.v["k"] == 0)
    sc_ref = T.scale.cpu().numpy().astype(np.float64)
    assert np.allclose(sc_ref, np.exp(T.raw["log_scale"].cpu().numpy().astype(np.float64)),
                       rtol=1e-6)
    T.step()
    # checkpoint round trip
    path = str(tmp_path / "ckpt.npz")
    T.save(path)
    T2 = tr.Trainer.from_scene(sc, cams, tgt, cfg)
    T2.load(path)
    for name in tr.PARAMS:
        assert torch.equal(T.raw[name], T2.raw[name]) and torch.equal(T.m[name], T2.m[name])
    assert torch.equal(T.sh16, T2.sh16) and torch.equal(T.opacity, T2.opacity)
    assert int(T2.step_dev.item()) == int(T.step_dev.item()) == 31
    T.step()
    T2.step()
    for name in tr.PARAMS:
        a, b = T.raw[name], T2.raw[name]
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6), name
