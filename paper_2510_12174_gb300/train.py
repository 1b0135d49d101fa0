"""Training step: render, the combined loss of Sec. 3.4, backward, Adam, and
the k-pruning of Sec. 3.3 - every stage in the library's kernels.

Parameters are kept as float32 master values in raw (pre-activation) form:
mean, quaternion, log-scale, logit-opacity, k, SH and logits.  The renderer
reads the activated scale and opacity that the fused Adam kernel writes after
each update, and bfloat16 copies of SH and logits when ``feat_bf16`` (the
mean, quaternion and k arrays are read in place).  Every ``prune_every``
steps the Gaussians with |k - 1| > T_k are removed (their order kept), k is
reset to 0.9 and its Adam moments to 0.

The paper does not print its learning rates (its supplementary table is not
available); the defaults are those of the 3DGS pipeline it builds on, with
one rate per array (SH included) and rates for the logits and k chosen in
the same range.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import abi
from . import rasterizer as rz

PARAMS = ("mean", "quat", "log_scale", "logit_opacity", "k", "sh", "sem")
# (activation, name of the renderer's array)
ACT = {"mean": abi.UNIGS_ACT_NONE, "quat": abi.UNIGS_ACT_NONE, "log_scale": abi.UNIGS_ACT_EXP,
       "logit_opacity": abi.UNIGS_ACT_SIGMOID, "k": abi.UNIGS_ACT_NONE,
       "sh": abi.UNIGS_ACT_NONE, "sem": abi.UNIGS_ACT_NONE}
GRAD_OF = {"mean": "mean", "quat": "quat", "log_scale": "scale", "logit_opacity": "opacity",
           "k": "kfac", "sh": "sh", "sem": "sem"}
# planar [planes][n] arrays, per-Gaussian vectors [n], and row-major [n][...] rows
LAYOUT = {"mean": "planes", "quat": "planes", "log_scale": "planes", "logit_opacity": "vec",
          "k": "vec", "sh": "rows", "sem": "rows"}


@dataclasses.dataclass
class TrainConfig:
    lr: Dict[str, float] = dataclasses.field(default_factory=lambda: {
        "mean": 1.6e-4, "quat": 1e-3, "log_scale": 5e-3, "logit_opacity": 5e-2, "k": 1e-3,
        "sh": 2.5e-3, "sem": 2.5e-3})
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    lam: Optional[Dict[str, float]] = None      # None: 1, 0.1, 0.1, 0.1, 0.1
    prune_every: int = 3000                     # K_p (Sec. 3.3)
    T_k: float = 0.2                            # threshold of the Tab. 6 ablation
    k_reset: float = 0.9
    feat_bf16: bool = True


def _raw_from_scene(scene, device) -> Dict[str, torch.Tensor]:
    f = lambda x: torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32)).to(device)
    op = np.clip(np.asarray(scene.opacity, dtype=np.float64), 1e-6, 1 - 1e-6)
    return {"mean": f(scene.mean), "quat": f(scene.quat),
            "log_scale": f(np.log(np.asarray(scene.scale, dtype=np.float64))),
            "logit_opacity": f(np.log(op / (1 - op))), "k": f(scene.kfac), "sh": f(scene.sh),
            "sem": f(scene.sem)}


class Trainer:
    """Owns master parameters, Adam state, the renderer and the targets."""

    def __init__(self, raw: Dict[str, torch.Tensor], sh_degree: int, cams: Sequence,
                 targets: Dict[str, torch.Tensor], cfg: Optional[TrainConfig] = None,
                 render_cfg: Optional[abi.unigs_config] = None):
        self.cfg = cfg or TrainConfig()
        self.cams = list(cams)
        self.sh_degree = int(sh_degree)
        self.device = raw["mean"].device
        self.raw = {k: raw[k].contiguous() for k in PARAMS}
        self.m = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.targets = targets
        self.render_cfg = render_cfg
        self.record = torch.zeros(abi.UNIGS_LOSS_RECORD_FLOATS, dtype=torch.float32,
                                  device=self.device)
        lam = abi.unigs_loss_lambda_default()
        for k, val in (self.cfg.lam or {}).items():
            setattr(lam, k, float(val))
        self.lam = lam
        self.hp = abi.unigs_adam_hparams(self.cfg.beta1, self.cfg.beta2, self.cfg.eps)
        self.steps_done = 0
        self._build()

    @staticmethod
    def from_scene(scene, cams, targets, cfg: Optional[TrainConfig] = None, device="cuda",
                   render_cfg=None) -> "Trainer":
        return Trainer(_raw_from_scene(scene, device), scene.sh_degree, cams, targets, cfg,
                       render_cfg)

    # ------------------------------------------------------------- buffers
    @property
    def n(self) -> int:
        return int(self.raw["mean"].shape[1])

    def _build(self):
        """Render copies, renderer, output and gradient buffers for the
        current Gaussian count (after construction, a prune or a load); the
        activated and bfloat16 copies are written by the library."""
        dev = self.device
        self.scale = torch.empty_like(self.raw["log_scale"])
        self.opacity = torch.empty_like(self.raw["logit_opacity"])
        if self.cfg.feat_bf16:
            self.sh16 = torch.empty(self.raw["sh"].shape, dtype=torch.bfloat16, device=dev)
            self.sem16 = torch.empty(self.raw["sem"].shape, dtype=torch.bfloat16, device=dev)
            sh, sem = self.sh16, self.sem16
        else:
            self.sh16 = self.sem16 = None
            sh, sem = self.raw["sh"], self.raw["sem"]
        self._copies()
        self.scene = rz.DeviceScene(self.raw["mean"], self.raw["quat"], self.scale, self.opacity,
                                    self.raw["k"], sh, sem, self.sh_degree)
        self.renderer = rz.Renderer(self.scene, self.cams, cfg=self.render_cfg)
        self.out = self.renderer.alloc_outputs()
        self.grads = self.renderer.alloc_grads()
        self.lgrad = self.renderer.alloc_loss_grads()
        self.g_depth_buf = torch.empty(self.renderer.n_pixels, dtype=torch.float32, device=dev)
        self._sized = False

    def _groups(self, with_grads: bool):
        groups = (abi.unigs_adam_group * len(PARAMS))()
        for i, name in enumerate(PARAMS):
            G = groups[i]
            x = self.raw[name]
            G.count = x.numel()
            G.activation = ACT[name]
            G.lr = float(self.cfg.lr[name])
            if G.count == 0:
                continue
            G.param = x.data_ptr()
            if with_grads:
                G.grad = self.grads[GRAD_OF[name]].data_ptr()
                G.m, G.v = self.m[name].data_ptr(), self.v[name].data_ptr()
            G.act_out = rz._ptr(self._act_out(name))
            G.bf16_out = rz._ptr(self._bf16_out(name))
        return groups

    def _copies(self):
        st = torch.cuda.current_stream(self.device).cuda_stream
        abi.check(abi.unigs_param_copies(self._groups(False), len(PARAMS), st),
                  "unigs_param_copies")

    def _act_out(self, name):
        return {"log_scale": self.scale, "logit_opacity": self.opacity}.get(name)

    def _bf16_out(self, name):
        return {"sh": self.sh16, "sem": self.sem16}.get(name)

    # ---------------------------------------------------------------- step
    def forward(self, readback: Optional[bool] = None):
        rb = (not self._sized) if readback is None else readback
        self.renderer.forward(self.out, readback=rb)
        self._sized = True
        return self.out

    def loss(self):
        """unigs_loss on the last forward; fills the loss gradients and the
        device record."""
        return self.renderer.loss(self.out, self.targets, self.record, self.lgrad, self.lam)

    def backward(self):
        up = {"rgb": self.lgrad["rgb"], "depth": self.lgrad["depth"],
              "normal_d": self.lgrad["normal_d"], "kmap": self.lgrad["kmap"],
              "logits": self.lgrad["logits"] if self.scene.n_sem else None}
        self.renderer.backward(self.out, up, grads=self.grads, g_depth_buf=self.g_depth_buf)
        return self.grads

    def adam(self):
        abi.check(abi.unigs_adam_step(self._groups(True), len(PARAMS), self.hp,
                                      self.step_dev.data_ptr(), self.renderer._stream()),
                  "unigs_adam_step")

    def step(self):
        """One training iteration; prunes every ``prune_every`` iterations.
        The loss stays on the device (``losses()`` reads it)."""
        self.forward()
        self.loss()
        self.backward()
        self.adam()
        self.steps_done += 1
        if self.cfg.prune_every and self.steps_done % self.cfg.prune_every == 0:
            self.prune()

    def losses(self) -> Dict[str, float]:
        r = self.record.cpu().numpy()
        return {"total": float(r[0]), "l1": float(r[1]), "normal": float(r[2]),
                "depth": float(r[3]), "seg": float(r[4]), "K": float(r[5])}

    # --------------------------------------------------------------- prune
    def prune(self) -> int:
        """Removes the Gaussians with |k - 1| > T_k; returns the survivors."""
        n = self.n
        st = self.renderer._stream()
        ws = torch.empty(max(abi.unigs_prune_workspace_bytes(n), 256), dtype=torch.uint8,
                         device=self.device)
        keep = ctypes.c_int64(0)
        abi.check(abi.unigs_prune_mark(self.raw["k"].data_ptr(), n, float(self.cfg.T_k),
                                       ws.data_ptr(), keep, st), "unigs_prune_mark")
        nk = int(keep.value)
        arrays = []
        new = {}

        def plan(name: str, src: torch.Tensor, fill=None):
            lay = LAYOUT[name]
            if lay == "planes":
                planes, row, shape = src.shape[0], 1, (src.shape[0], nk)
            elif lay == "vec":
                planes, row, shape = 1, 1, (nk,)
            else:
                planes, row, shape = 1, int(np.prod(src.shape[1:])), (nk,) + tuple(src.shape[1:])
            dst = torch.empty(shape, dtype=src.dtype, device=self.device)
            a = abi.unigs_prune_array()
            a.src = src.data_ptr() if src.numel() else None
            a.dst = dst.data_ptr() if dst.numel() else None
            a.planes, a.row, a.elem_bytes = planes, row, src.element_size()
            if fill is not None:
                a.fill, a.fill_value = 1, float(fill)
            arrays.append(a)
            return dst

        for name in PARAMS:
            reset = name == "k"
            new[("raw", name)] = plan(name, self.raw[name], self.cfg.k_reset if reset else None)
            new[("m", name)] = plan(name, self.m[name], 0.0 if reset else None)
            new[("v", name)] = plan(name, self.v[name], 0.0 if reset else None)
        arr = (abi.unigs_prune_array * len(arrays))(*arrays)
        abi.check(abi.unigs_prune_compact(arr, len(arrays), n, nk, ws.data_ptr(), st),
                  "unigs_prune_compact")
        for name in PARAMS:
            self.raw[name] = new[("raw", name)]
            self.m[name] = new[("m", name)]
            self.v[name] = new[("v", name)]
        self._build()
        return nk

    # ---------------------------------------------------------- checkpoint
    def state(self) -> Dict[str, np.ndarray]:
        d = {}
        for name in PARAMS:
            d["raw/" + name] = self.raw[name].cpu().numpy()
            d["m/" + name] = self.m[name].cpu().numpy()
            d["v/" + name] = self.v[name].cpu().numpy()
        d["step"] = self.step_dev.cpu().numpy()
        d["steps_done"] = np.array([self.steps_done], dtype=np.int64)
        d["sh_degree"] = np.array([self.sh_degree], dtype=np.int64)
        return d

    def save(self, path: str) -> None:
        np.savez(path, **self.state())

    def load(self, path: str) -> None:
        z = np.load(path)
        for name in PARAMS:
            self.raw[name] = torch.as_tensor(z["raw/" + name]).to(self.device).contiguous()
            self.m[name] = torch.as_tensor(z["m/" + name]).to(self.device).contiguous()
            self.v[name] = torch.as_tensor(z["v/" + name]).to(self.device).contiguous()
        self.step_dev.copy_(torch.as_tensor(z["step"]).to(self.device))
        self.steps_done = int(z["steps_done"][0])
        self.sh_degree = int(z["sh_degree"][0])
        self._build()
