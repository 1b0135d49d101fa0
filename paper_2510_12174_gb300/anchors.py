"""Anchor sets on the device and their decode into the rasterizer's Gaussians
(include/unigs_anchors.h: the MLP attribute prediction of Sec. 3.1).

Argument marshalling only: the MLPs and their backward run in the library's
kernels (csrc/anchors.cu).
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np
import torch

from . import abi
from .rasterizer import DeviceScene


def _ptr(x: Optional[torch.Tensor]):
    return None if x is None else x.data_ptr()


class DeviceAnchors:
    """An anchor set as CUDA tensors: pos [3][A], scale [3][A], offsets
    [A][M][3], feat [A][F], sem [A][C], kfac [A] and, per MLP name in
    abi.ANCHOR_MLPS, w1 [H][F], b1 [H], w2 [out][H], b2 [out] (float32)."""

    def __init__(self, pos, scale, offsets, feat, sem, kfac, mlps: Dict[str, Dict[str, torch.Tensor]]):
        self.pos, self.scale, self.offsets, self.feat = pos, scale, offsets, feat
        self.sem, self.kfac, self.mlps = sem, kfac, mlps

    @staticmethod
    def from_arrays(arrs: Dict[str, np.ndarray], mlps: Dict[str, Dict[str, np.ndarray]],
                    device="cuda") -> "DeviceAnchors":
        """From row-per-anchor arrays (pos, scale [A,3], offsets [A,M,3],
        feat [A,F], sem [A,C], kfac [A]) and the MLP parameter arrays."""
        t = lambda x: torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32)).to(device)
        return DeviceAnchors(t(np.asarray(arrs["pos"]).T), t(np.asarray(arrs["scale"]).T),
                             t(arrs["offsets"]), t(arrs["feat"]), t(arrs["sem"]), t(arrs["kfac"]),
                             {n: {k: t(v) for k, v in mlps[n].items()} for n in abi.ANCHOR_MLPS
                              if n in mlps})

    @property
    def n(self) -> int:
        return int(self.feat.shape[0])

    @property
    def n_offsets(self) -> int:
        return int(self.offsets.shape[1])

    @property
    def n_sem(self) -> int:
        return int(self.sem.shape[1])

    def struct(self) -> abi.unigs_anchors:
        a = abi.unigs_anchors()
        a.n, a.n_offsets = self.n, self.n_offsets
        a.feat_dim, a.hidden, a.n_sem = int(self.feat.shape[1]), abi.UNIGS_ANCHOR_HIDDEN, self.n_sem
        if "k" in self.mlps:
            a.hidden = int(self.mlps["k"]["w1"].shape[0])
        a.pos, a.scale, a.offsets = _ptr(self.pos), _ptr(self.scale), _ptr(self.offsets)
        a.feat, a.sem, a.kfac = _ptr(self.feat), _ptr(self.sem) if self.n_sem else None, \
            _ptr(self.kfac)
        for n in abi.ANCHOR_MLPS:
            if n not in self.mlps:
                continue
            m = getattr(a, "mlp_" + n)
            for k in ("w1", "b1", "w2", "b2"):
                setattr(m, k, _ptr(self.mlps[n][k]))
        return a

    def decode(self, feat_bf16: bool = False, out: Optional[DeviceScene] = None) -> DeviceScene:
        """The anchors' Gaussians (N = A M, SH degree 0) as a DeviceScene."""
        dev = self.feat.device
        N, C = self.n * self.n_offsets, self.n_sem
        if out is None:
            ft = torch.bfloat16 if feat_bf16 else torch.float32
            e = lambda *s, dt=torch.float32: torch.empty(*s, dtype=dt, device=dev)
            out = DeviceScene(e(3, N), e(4, N), e(3, N), e(N), e(N), e(N, 1, 3, dt=ft),
                              e(N, C, dt=ft), 0)
        g = abi.unigs_anchor_gaussians()
        g.mean, g.quat, g.scale = _ptr(out.mean), _ptr(out.quat), _ptr(out.scale)
        g.opacity, g.kfac, g.sh = _ptr(out.opacity), _ptr(out.kfac), _ptr(out.sh)
        g.sem = _ptr(out.sem) if C else None
        g.feat_dtype = 1 if out.sh.dtype == torch.bfloat16 else 0
        abi.check(abi.unigs_anchor_decode(self.struct(), g,
                                          torch.cuda.current_stream(dev).cuda_stream),
                  "unigs_anchor_decode")
        return out

    def alloc_grads(self) -> Dict:
        z = torch.zeros_like
        return {"pos": z(self.pos), "scale": z(self.scale), "offsets": z(self.offsets),
                "feat": z(self.feat), "sem": z(self.sem), "kfac": z(self.kfac),
                "mlps": {n: {k: z(v) for k, v in d.items()} for n, d in self.mlps.items()}}

    def decode_backward(self, gauss_grads: Dict[str, torch.Tensor], grads: Optional[Dict] = None,
                        accumulate: bool = False) -> Dict:
        """dL/d(anchor arrays, MLP parameters) from the decoded Gaussians'
        parameter gradients (Renderer.backward's dict)."""
        dev = self.feat.device
        grads = grads if grads is not None else self.alloc_grads()
        pg = abi.unigs_param_grads()
        for k in ("mean", "quat", "scale", "opacity", "kfac", "sh", "sem"):
            v = gauss_grads.get(k)
            setattr(pg, k, _ptr(v) if v is not None and v.numel() else None)
        o = abi.unigs_anchor_grads()
        for k in ("pos", "scale", "offsets", "feat", "kfac"):
            setattr(o, k, _ptr(grads[k]))
        o.sem = _ptr(grads["sem"]) if self.n_sem else None
        for n in abi.ANCHOR_MLPS:
            if n not in grads["mlps"]:
                continue
            m = getattr(o, "mlp_" + n)
            for k in ("w1", "b1", "w2", "b2"):
                setattr(m, k, _ptr(grads["mlps"][n][k]))
        o.accumulate = 1 if accumulate else 0
        abi.check(abi.unigs_anchor_decode_bwd(self.struct(), pg, o,
                                              torch.cuda.current_stream(dev).cuda_stream),
                  "unigs_anchor_decode_bwd")
        return grads
