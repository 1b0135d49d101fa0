"""FP64 oracle of the anchor attribute prediction (Sec. 3.1, Fig. 2 (a)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

An anchor carries a position x, a positive scale l, M learnable offsets O_m
(in units of l), a feature f, base semantic logits o_ah and a base gradient
factor k_ah.  Two-layer perceptrons MLP(f) = W2 relu(W1 f + b1) + b2 predict,
from the feature alone, the attributes of the anchor's M Gaussians:

* semantic logits (the paper's Repeat(o_ah, M) (x) sigma(MLP_o(f))):
  o_m = o_ah * sigma(MLP_o(f)), MLP_o: R^F -> R^C, the same for every m;
* gradient factor: k_m = k_ah * sigma(MLP_k(f)), MLP_k: R^F -> R;
* opacity: alpha_m = sigma(MLP_alpha(f)_m), MLP_alpha: R^F -> R^M;
* colour: c_m = sigma(MLP_c(f)_{3m..3m+2}), MLP_c: R^F -> R^(3M), stored as
  the degree-0 SH coefficient h_m = (c_m - 1/2) / Y_00, so that the renderer's
  colour Y_00 h + 1/2 equals c_m;
* covariance: MLP_cov: R^F -> R^(7M); scale s_m = l * sigma(first 3 of the
  m-th 7), rotation q_m = the last 4 (the renderer normalises it);
* position: mu_m = x + l * O_m.

Gaussian g = a M + m is child m of anchor a.  The derivative is taken by
autograd (the tests pin it by finite differences and closed forms).
"""
from __future__ import annotations

import dataclasses
from typing import Dict

import numpy as np
import torch

F64 = torch.float64
Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)), the degree-0 real SH basis
MLP_NAMES = ("sem", "k", "opacity", "color", "cov")


def mlp_out_dims(n_sem: int, n_offsets: int) -> Dict[str, int]:
    """Output width of each branch."""
    return {"sem": n_sem, "k": 1, "opacity": n_offsets, "color": 3 * n_offsets,
            "cov": 7 * n_offsets}


@dataclasses.dataclass
class Anchors:
    """float64 leaves (optionally requiring grad)."""
    pos: torch.Tensor      # [A,3]
    scale: torch.Tensor    # [A,3], positive
    offsets: torch.Tensor  # [A,M,3]
    feat: torch.Tensor     # [A,F]
    sem: torch.Tensor      # [A,C]
    kfac: torch.Tensor     # [A]
    mlps: Dict[str, Dict[str, torch.Tensor]]  # name -> {w1 [H,F], b1 [H], w2 [O,H], b2 [O]}

    @staticmethod
    def from_arrays(arrs: Dict[str, np.ndarray], mlps: Dict[str, Dict[str, np.ndarray]],
                    requires_grad: bool = False) -> "Anchors":
        t = lambda x: torch.as_tensor(np.asarray(x, dtype=np.float64)).requires_grad_(requires_grad)
        return Anchors(t(arrs["pos"]), t(arrs["scale"]), t(arrs["offsets"]), t(arrs["feat"]),
                       t(arrs["sem"]), t(arrs["kfac"]),
                       {n: {k: t(v) for k, v in mlps[n].items()} for n in MLP_NAMES
                        if n in mlps})

    def leaves(self):
        out = [self.pos, self.scale, self.offsets, self.feat, self.sem, self.kfac]
        for n in MLP_NAMES:
            if n in self.mlps:
                out += [self.mlps[n][k] for k in ("w1", "b1", "w2", "b2")]
        return out


def mlp(p: Dict[str, torch.Tensor], f: torch.Tensor) -> torch.Tensor:
    """W2 relu(W1 f + b1) + b2 for every row of f [A,F]."""
    h = torch.relu(f @ p["w1"].T + p["b1"])
    return h @ p["w2"].T + p["b2"]


def decode(a: Anchors) -> Dict[str, torch.Tensor]:
    """The M Gaussians of every anchor, in the renderer's layouts: mean [3,N],
    quat [4,N], scale [3,N], opacity [N], kfac [N], sh [N,1,3], sem [N,C]."""
    A, M = a.offsets.shape[0], a.offsets.shape[1]
    sig = torch.sigmoid
    y = {n: mlp(a.mlps[n], a.feat) for n in MLP_NAMES if n in a.mlps}
    mean = a.pos[:, None, :] + a.scale[:, None, :] * a.offsets             # [A,M,3]
    cov = y["cov"].reshape(A, M, 7)
    scale = a.scale[:, None, :] * sig(cov[..., :3])                          # [A,M,3]
    quat = cov[..., 3:]                                                       # [A,M,4]
    opacity = sig(y["opacity"])                                               # [A,M]
    color = sig(y["color"].reshape(A, M, 3))
    sh = ((color - 0.5) / Y00).reshape(A * M, 1, 3)
    C = a.sem.shape[1]
    sem = (a.sem * sig(y["sem"]) if C else a.sem)[:, None, :].expand(A, M, C)
    kfac = (a.kfac * sig(y["k"][:, 0]))[:, None].expand(A, M)
    N = A * M
    return {"mean": mean.reshape(N, 3).T, "quat": quat.reshape(N, 4).T,
            "scale": scale.reshape(N, 3).T, "opacity": opacity.reshape(N),
            "kfac": kfac.reshape(N), "sh": sh, "sem": sem.reshape(N, -1)}


def decode_and_grad(arrs, mlps, upstream: Dict[str, np.ndarray]):
    """Decoded Gaussians and the exact gradients of L = sum <out, upstream>
    with respect to every anchor array and MLP parameter."""
    a = Anchors.from_arrays(arrs, mlps, requires_grad=True)
    out = decode(a)
    loss = torch.zeros((), dtype=F64)
    for k, v in out.items():
        loss = loss + (v * torch.as_tensor(np.asarray(upstream[k], dtype=np.float64))
                       .reshape(v.shape)).sum()
    loss.backward()
    g = {"pos": a.pos.grad, "scale": a.scale.grad, "offsets": a.offsets.grad,
         "feat": a.feat.grad, "sem": a.sem.grad, "kfac": a.kfac.grad}
    gm = {n: {k: a.mlps[n][k].grad for k in ("w1", "b1", "w2", "b2")} for n in a.mlps}
    g = {k: (v if v is not None else torch.zeros_like(getattr(a, k))) for k, v in g.items()}
    return ({k: v.detach().numpy() for k, v in out.items()},
            {k: v.numpy() for k, v in g.items()},
            {n: {k: v.numpy() for k, v in d.items()} for n, d in gm.items()})
