"""Pins of the training-step oracle (oracle/train.py) to closed forms, library
routines and finite differences - nothing here re-types the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import train as ot


def _maps(rng, shapes, C=5):
    out = {"rgb": [], "depth": [], "normal_d": [], "kmap": [], "logits": []}
    tgt = {"rgb": [], "depth": [], "normal": [], "label": []}
    for (H, W) in shapes:
        out["rgb"].append(rng.uniform(0, 1, (3, H, W)))
        out["depth"].append(rng.uniform(1, 3, (H, W)))
        n = rng.normal(size=(3, H, W))
        out["normal_d"].append(n / np.linalg.norm(n, axis=0))
        out["kmap"].append(rng.uniform(0.5, 1.5, (H, W)))
        out["logits"].append(rng.normal(size=(C, H, W)))
        tgt["rgb"].append(rng.uniform(0, 1, (3, H, W)))
        d = rng.uniform(1, 3, (H, W))
        d[rng.uniform(size=(H, W)) < 0.2] = 0.0          # missing measurements
        tgt["depth"].append(d)
        n = rng.normal(size=(3, H, W))
        tgt["normal"].append(n / np.linalg.norm(n, axis=0))
        lab = rng.integers(0, C, (H, W))
        lab[rng.uniform(size=(H, W)) < 0.1] = -1           # unlabelled
        tgt["label"].append(lab)
    return out, tgt


def test_l1_depth_K_closed_forms():
    shapes = [(4, 5), (3, 2)]
    P = 26
    out = {"rgb": [np.full((3,) + s, 0.5) for s in shapes],
           "depth": [np.full(s, 2.0) for s in shapes],
           "normal_d": [np.zeros((3,) + s) for s in shapes],
           "kmap": [np.full(s, 0.9) for s in shapes],
           "logits": [np.zeros((4,) + s) for s in shapes]}
    dt = [np.full(s, 2.5) for s in shapes]
    dt[1][:] = 0.0                                        # second view: no depth
    tgt = {"rgb": [np.full((3,) + s, 0.25) for s in shapes], "depth": dt,
           "normal": [np.zeros((3,) + s) for s in shapes],
           "label": [np.zeros(s, dtype=np.int64) for s in shapes]}
    r = ot.loss_terms(out, tgt)
    assert r["l1"][0] == pytest.approx(0.25)
    assert np.all(r["l1"][1]["rgb"][0] == 1.0 / (3 * P))
    assert r["depth"][0] == pytest.approx(0.5)
    assert np.all(r["depth"][1]["depth"][0] == -1.0 / 20)
    assert np.all(r["depth"][1]["depth"][1] == 0.0)
    assert r["K"][0] == pytest.approx(0.1)
    assert np.all(r["K"][1]["kmap"][1] == -1.0 / P)
    # uniform logits: cross-entropy log C at every labelled pixel
    assert r["seg"][0] == pytest.approx(math.log(4))
    # zero predicted normals (invalid pixels): cosine loss 1
    assert r["normal"][0] == pytest.approx(1.0)


def test_cosine_loss_special_cases():
    rng = np.random.default_rng(1)
    out, tgt = _maps(rng, [(6, 7)])
    out["normal_d"] = [n.copy() for n in tgt["normal"]]
    assert ot.loss_terms(out, tgt)["normal"][0] == pytest.approx(0.0, abs=1e-12)
    out["normal_d"] = [-n for n in tgt["normal"]]
    r = ot.loss_terms(out, tgt)["normal"]
    assert r[0] == pytest.approx(2.0)
    assert np.allclose(r[1]["normal_d"][0], -tgt["normal"][0] / 42)


def test_cross_entropy_matches_library_routine():
    rng = np.random.default_rng(2)
    out, tgt = _maps(rng, [(5, 6), (4, 3)], C=7)
    r = ot.loss_terms(out, tgt)["seg"]
    O = torch.tensor(np.concatenate([o.reshape(7, -1) for o in out["logits"]], 1).T,
                     requires_grad=True)
    lab = torch.tensor(np.concatenate([l.ravel() for l in tgt["label"]]))
    ref = torch.nn.functional.cross_entropy(O, lab, ignore_index=-1)
    ref.backward()
    assert r[0] == pytest.approx(ref.item(), rel=1e-12)
    g = np.concatenate([x.reshape(7, -1) for x in r[1]["logits"]], 1).T
    assert np.allclose(g, O.grad.numpy(), rtol=1e-12, atol=1e-15)
    # rows of (softmax - onehot) sum to zero
    assert np.allclose(g.sum(1), 0, atol=1e-15)


def test_combined_total_and_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    out, tgt = _maps(rng, [(5, 4), (3, 6)])
    terms = ot.loss_terms(out, tgt)
    total, w, grads = ot.combine(terms)
    l1 = terms["l1"][0]
    # every term weighted to 0.1 |L_l1|: closed form of the total
    assert total == pytest.approx(l1 * (1 + 0.1 * 4))
    assert w["seg"] == pytest.approx(0.1 * l1 / terms["seg"][0])

    def frozen(o):
        t = ot.loss_terms(o, tgt)
        return sum(w[k] * t[k][0] for k in ot.TERMS)

    h = 1e-6
    for key in ("rgb", "depth", "normal_d", "kmap", "logits"):
        for _ in range(4):
            cam = int(rng.integers(0, 2))
            idx = tuple(int(rng.integers(0, s)) for s in out[key][cam].shape)
            plus = {k: [a.copy() for a in v] for k, v in out.items()}
            minus = {k: [a.copy() for a in v] for k, v in out.items()}
            plus[key][cam][idx] += h
            minus[key][cam][idx] -= h
            fd = (frozen(plus) - frozen(minus)) / (2 * h)
            assert grads[key][cam][idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (key, idx)


def test_zero_term_gets_zero_weight():
    rng = np.random.default_rng(4)
    out, tgt = _maps(rng, [(3, 3)])
    tgt["depth"] = [np.zeros((3, 3))]
    terms = ot.loss_terms(out, tgt)
    total, w, grads = ot.combine(terms)
    assert terms["depth"][0] == 0.0 and w["depth"] == 0.0
    assert np.all(grads["depth"][0] == 0.0)


def test_adam_first_step_and_library_routine():
    rng = np.random.default_rng(5)
    raw = rng.normal(size=50)
    g = rng.normal(size=50)
    lr = 1e-2
    r1, m, v, a = ot.adam_step(raw, g, np.zeros(50), np.zeros(50), 1, lr, eps=1e-15)
    # bias-corrected first step: lr * sign(g)
    assert np.allclose(raw - r1, lr * np.sign(g), rtol=1e-12)
    # several steps against torch.optim.Adam (same eps, no weight decay)
    p = torch.tensor(raw, requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    x, m, v = raw.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        gt = rng.normal(size=50)
        p.grad = torch.tensor(gt)
        opt.step()
        x, m, v, _ = ot.adam_step(x, gt, m, v, t, lr, eps=1e-8)
    assert np.allclose(x, p.detach().numpy(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("act", [ot.ACT_EXP, ot.ACT_SIGMOID])
def test_adam_activation_chain(act):
    """The raw-space gradient is the activated-space gradient times f'(raw):
    the first moment after one step from zero equals (1 - beta1) g f'(raw),
    with f' taken by central differences."""
    rng = np.random.default_rng(6)
    raw = rng.normal(size=20)
    g = rng.normal(size=20)
    _, m, _, a = ot.adam_step(raw, g, np.zeros(20), np.zeros(20), 1, 1e-3, act=act)
    h = 1e-6
    fp = (ot.activate(raw + h, act) - ot.activate(raw - h, act)) / (2 * h)
    assert np.allclose(m, 0.1 * g * fp, rtol=1e-8)
    ref = np.exp(raw) if act == ot.ACT_EXP else 1 / (1 + np.exp(-raw))
    assert np.allclose(ot.activate(raw, act), ref)


def test_prune_rule_hand_case():
    k = np.array([1.0, 1.1, 1.3, 0.85, 0.7, 0.9, 1.25, 0.79], dtype=np.float32)
    keep = ot.prune_mask(k, 0.2)
    assert keep.tolist() == [True, True, False, True, False, True, False, False]


def test_out_of_range_labels_are_unlabelled():
    rng = np.random.default_rng(7)
    out, tgt = _maps(rng, [(4, 4)], C=3)
    ref = ot.loss_terms(out, tgt)["seg"][0]
    tgt2 = {k: [a.copy() for a in v] for k, v in tgt.items()}
    lab = tgt2["label"][0]
    lab[lab == -1] = 3                    # the same pixels, marked by an out-of-range id
    r = ot.loss_terms(out, tgt2)["seg"]
    assert r[0] == pytest.approx(ref, rel=1e-15)
    assert np.all(r[1]["logits"][0][:, lab == 3] == 0)
