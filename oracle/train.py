"""FP64 oracle of the training step around the rasterizer.

TEST INFRASTRUCTURE ONLY (see the package header): the plain definitions that
the CUDA loss, optimizer and pruning kernels are checked against.

* :func:`loss_terms` - the five loss terms of the combined objective of the
  Loss Function paragraph of Sec. 3.4 (SSIM omitted), each as a value and its
  exact gradient with respect to the rendered maps:
  L_l1 (RGB), L_normal = 1 - mean cosine (Eq. csloss with the mean over the
  pixel set Omega written out in the supplementary, whose gradient is
  -N_target / |Omega|, Eq. gradientn), L_depth (L1 on depth), L_seg
  (cross-entropy of the rendered logits, Eq. semantic_render and the text
  after it) and L_K = ||K - 1||_1 (Sec. 3.3, Gradient Factor Rasterization).
* :func:`combine` - the magnitude-normalised sum
  L_all = l1 * L_l1 + sum_i l_i * |L_l1| * L_i / |L_i|; the factors
  |L_l1| / |L_i| are constants of the step (weights, not differentiated).
* :func:`adam_step` - one Adam update of a raw (pre-activation) parameter from
  the gradient of its activated value, with the activated float32 value and
  its bfloat16 copy the renderer reads.
* :func:`prune_mask` - the pruning rule of Sec. 3.3: drop Gaussians with
  |k - 1| > T_k; survivors keep their order and k is reset to 0.9.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

TERMS = ("l1", "normal", "depth", "seg", "K")
# Loss Function paragraph, Sec. 3.4: lambda_1 = 1, every other lambda 0.1
# (lambda_2 weighs SSIM, which this objective omits).
DEFAULT_LAMBDA = {"l1": 1.0, "normal": 0.1, "depth": 0.1, "seg": 0.1, "K": 0.1}

ACT_NONE, ACT_EXP, ACT_SIGMOID = 0, 1, 2


def _cat(maps: Sequence[np.ndarray], channels: int) -> np.ndarray:
    """Per-camera maps [C][H][W] (or [H][W]) -> [C, pixels of all cameras]."""
    return np.concatenate([np.asarray(m, dtype=np.float64).reshape(channels, -1)
                           for m in maps], axis=1)


def loss_terms(out: Dict[str, List[np.ndarray]], tgt: Dict[str, List[np.ndarray]]):
    """Values and gradients of the five terms over the pixels of all cameras.

    out: per-camera lists 'rgb' [3,H,W], 'depth' [H,W], 'normal_d' [3,H,W],
    'kmap' [H,W], 'logits' [C,H,W].  tgt: 'rgb' [3,H,W], 'depth' [H,W] (<= 0:
    no measurement, excluded), 'normal' [3,H,W], 'label' [H,W] int (outside
    [0, C): unlabelled, excluded).  Returns {term: (value, {map: gradient list})}.
    """
    shapes = [np.asarray(d).shape for d in out["depth"]]
    P = sum(int(np.prod(s)) for s in shapes)

    def split(flat, channels):
        res, a = [], 0
        for s in shapes:
            n = int(np.prod(s))
            res.append(flat[:, a:a + n].reshape((channels,) + s) if channels > 1
                       else flat[0, a:a + n].reshape(s))
            a += n
        return res

    res = {}
    # L1 on RGB: mean over the 3P entries
    d = _cat(out["rgb"], 3) - _cat(tgt["rgb"], 3)
    res["l1"] = (np.abs(d).sum() / (3 * P), {"rgb": split(np.sign(d) / (3 * P), 3)})
    # cosine normal loss over Omega = every pixel
    N = _cat(out["normal_d"], 3)
    Nt = _cat(tgt["normal"], 3)
    res["normal"] = (1.0 - (N * Nt).sum() / P, {"normal_d": split(-Nt / P, 3)})
    # L1 on depth over the pixels with a measurement
    D = _cat(out["depth"], 1)[0]
    Dt = _cat(tgt["depth"], 1)[0]
    valid = Dt > 0
    nv = int(valid.sum())
    gD = np.zeros(P)
    if nv:
        dd = D - Dt
        val = np.abs(dd[valid]).sum() / nv
        gD[valid] = np.sign(dd[valid]) / nv
    else:
        val = 0.0
    res["depth"] = (val, {"depth": split(gD[None], 1)})
    # cross-entropy of the rendered logits over the labelled pixels
    O = _cat(out["logits"], np.asarray(out["logits"][0]).shape[0])
    C = O.shape[0]
    lab = np.concatenate([np.asarray(l).reshape(-1) for l in tgt["label"]]).astype(np.int64)
    has = (lab >= 0) & (lab < C)
    nl = int(has.sum())
    gO = np.zeros_like(O)
    if nl:
        mx = O.max(axis=0)
        e = np.exp(O - mx)
        Z = e.sum(axis=0)
        lse = mx + np.log(Z)
        idx = np.where(has)[0]
        val = (lse[idx] - O[lab[idx], idx]).sum() / nl
        p = e / Z
        gO[:, idx] = p[:, idx]
        gO[lab[idx], idx] -= 1.0
        gO /= nl
    else:
        val = 0.0
    res["seg"] = (val, {"logits": split(gO, C)})
    # L_K = ||K - 1||_1, as a mean over pixels
    K = _cat(out["kmap"], 1)[0]
    res["K"] = (np.abs(K - 1.0).sum() / P, {"kmap": split(np.sign(K - 1.0)[None] / P, 1)})
    return res


def combine(terms, lam: Dict[str, float] = DEFAULT_LAMBDA):
    """(L_all, weights, upstream gradients) of the magnitude-normalised sum."""
    l1 = terms["l1"][0]
    w = {"l1": lam["l1"]}
    for t in TERMS[1:]:
        v = terms[t][0]
        w[t] = lam[t] * abs(l1) / abs(v) if v != 0 else 0.0
    total = sum(w[t] * terms[t][0] for t in TERMS)
    grads: Dict[str, List[np.ndarray]] = {}
    for t in TERMS:
        for k, gl in terms[t][1].items():
            scaled = [w[t] * g for g in gl]
            grads[k] = scaled if k not in grads else [a + b for a, b in zip(grads[k], scaled)]
    return total, w, grads


def activate(raw: np.ndarray, act: int) -> np.ndarray:
    raw = np.asarray(raw, dtype=np.float64)
    if act == ACT_EXP:
        return np.exp(raw)
    if act == ACT_SIGMOID:
        return 1.0 / (1.0 + np.exp(-raw))
    return raw.copy()


def adam_step(raw, grad_act, m, v, t: int, lr: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-15, act: int = ACT_NONE):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) on the raw parameter.

    The gradient arrives for the activated value a = f(raw) the renderer read
    (exp for scales, sigmoid for opacity, identity otherwise) and is taken
    back through f' first.  Returns (raw, m, v, activated value)."""
    raw = np.asarray(raw, dtype=np.float64)
    a = activate(raw, act)
    g = np.asarray(grad_act, dtype=np.float64)
    if act == ACT_EXP:
        g = g * a
    elif act == ACT_SIGMOID:
        g = g * a * (1.0 - a)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    raw = raw - lr * mhat / (np.sqrt(vhat) + eps)
    return raw, m, v, activate(raw, act)


def prune_mask(k_raw: np.ndarray, T_k: float) -> np.ndarray:
    """Keep flags of the pruning rule: |k - 1| <= T_k.  The comparison is a
    discrete decision and is taken in float32, the precision of k."""
    k = np.asarray(k_raw, dtype=np.float32)
    return ~(np.abs(k - np.float32(1.0)) > np.float32(T_k))
