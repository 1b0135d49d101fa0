"""Python front end of libunigs: device buffers, call sequencing, autograd.

PyTorch supplies device memory, the current CUDA stream and autograd; every
stage of the rasterizer runs in the library's kernels through :mod:`abi`.
There is no CPU fallback: without the built library or a CUDA device the
calls raise.

Images of several cameras are returned concatenated ("flat"): camera k's block
of a C-channel output starts at element C * pixel_offset[k] and is laid out
[C][H_k][W_k]; :meth:`Renderer.split` cuts a flat output into per-camera views.
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import abi

OUT_CHANNELS = {"rgb": 3, "depth": 1, "normal_g": 3, "kmap": 1, "T_final": 1, "normal_d": 3}


def make_cameras(cams) -> ctypes.Array:
    """ctypes array of unigs_camera from objects with the Camera fields."""
    arr = (abi.unigs_camera * len(cams))()
    for k, c in enumerate(cams):
        a = arr[k]
        a.width, a.height = int(c.width), int(c.height)
        a.fx, a.fy, a.cx, a.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        for name in ("R_wc", "t_wc", "R_cw", "C"):
            vals = np.asarray(getattr(c, name), dtype=np.float32).ravel()
            getattr(a, name)[:] = [float(v) for v in vals]
        a.z_near = float(c.z_near)
    return arr


class DeviceScene:
    """Gaussian parameters as CUDA tensors in the library's layout."""

    def __init__(self, mean, quat, scale, opacity, kfac, sh, sem, sh_degree: int):
        self.mean, self.quat, self.scale = mean, quat, scale
        self.opacity, self.kfac, self.sh, self.sem = opacity, kfac, sh, sem
        self.sh_degree = int(sh_degree)

    @staticmethod
    def from_scene(scene, device="cuda", feat_bf16: Optional[bool] = None) -> "DeviceScene":
        bf16 = scene.feat_bf16 if feat_bf16 is None else feat_bf16
        ft = torch.bfloat16 if bf16 else torch.float32

        def t(x, dt=torch.float32):
            return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).to(
                device=device, dtype=dt).contiguous()

        return DeviceScene(t(scene.mean), t(scene.quat), t(scale_of(scene)), t(scene.opacity),
                           t(scene.kfac), t(scene.sh, ft), t(scene.sem, ft), scene.sh_degree)

    @property
    def n(self) -> int:
        return int(self.mean.shape[1])

    @property
    def n_sem(self) -> int:
        return int(self.sem.shape[1])

    @property
    def feat_dtype(self) -> int:
        return 1 if self.sh.dtype == torch.bfloat16 else 0

    def tensors(self):
        return [self.mean, self.quat, self.scale, self.opacity, self.kfac, self.sh, self.sem]

    def struct(self) -> abi.unigs_gaussians:
        g = abi.unigs_gaussians()
        g.n = self.n
        g.sh_degree = self.sh_degree
        g.n_sem = self.n_sem
        g.feat_dtype = self.feat_dtype
        for name in ("mean", "quat", "scale", "opacity", "kfac", "sh", "sem"):
            x = getattr(self, name)
            assert x.is_cuda and x.is_contiguous(), name
            setattr(g, name, x.data_ptr() if x.numel() else None)
        return g


def scale_of(scene):
    return scene.scale


def _ptr(x: Optional[torch.Tensor]):
    return None if x is None else x.data_ptr()


class Renderer:
    """Plans, owns the workspace and runs the forward / backward sequences.

    ``capacity`` bounds the (tile, Gaussian) instances; with ``grow`` the
    per-call path reads the instance count back and re-plans when it is
    exceeded.  ``graph_safe`` sequences never synchronise (capture them in a
    CUDA graph); an overflow then shows in :meth:`status`.
    """

    def __init__(self, scene: DeviceScene, cams, cfg: Optional[abi.unigs_config] = None,
                 capacity: int = 0, center_depth: bool = False):
        self.scene = scene
        self.cam_list = list(cams)
        self.cams = make_cameras(self.cam_list)
        self.cfg = cfg if cfg is not None else abi.unigs_config_default()
        if center_depth:
            self.cfg.flags |= abi.UNIGS_FLAG_CENTER_DEPTH
        self.device = scene.mean.device
        self.last_instances = None
        self._plan(capacity)

    # ------------------------------------------------------------------ plan
    def _plan(self, capacity: int):
        self.plan = abi.unigs_plan()
        g = self.scene.struct()
        abi.check(abi.unigs_plan_init(self.plan, g, self.cams, len(self.cam_list), self.cfg,
                                      int(capacity)), "unigs_plan_init")
        nbytes = abi.unigs_workspace_bytes(self.plan)
        self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        self.n_pixels = int(self.plan.n_pixels)

    @property
    def capacity(self) -> int:
        return int(self.plan.capacity)

    def pixel_offsets(self) -> List[int]:
        return [int(self.plan.pixel_offset[k]) for k in range(len(self.cam_list) + 1)]

    def split(self, flat: torch.Tensor, channels: int) -> List[torch.Tensor]:
        offs = self.pixel_offsets()
        views = []
        for k, c in enumerate(self.cam_list):
            a, b = offs[k] * channels, offs[k + 1] * channels
            shape = (channels, c.height, c.width) if channels > 1 else (c.height, c.width)
            views.append(flat[a:b].view(shape))
        return views

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def alloc_outputs(self) -> Dict[str, torch.Tensor]:
        P = self.n_pixels
        f = lambda c: torch.empty(c * P, dtype=torch.float32, device=self.device)
        out = {k: f(c) for k, c in OUT_CHANNELS.items()}
        out["logits"] = f(self.scene.n_sem) if self.scene.n_sem else f(0)
        out["n_contrib"] = torch.empty(P, dtype=torch.int32, device=self.device)
        return out

    def _out_struct(self, out) -> abi.unigs_outputs:
        o = abi.unigs_outputs()
        o.rgb, o.depth, o.normal_g = _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["normal_g"])
        o.kmap, o.T_final, o.n_contrib = _ptr(out["kmap"]), _ptr(out["T_final"]), _ptr(out["n_contrib"])
        o.logits = _ptr(out["logits"]) if self.scene.n_sem else None
        return o

    # --------------------------------------------------------------- forward
    def preprocess_and_sort(self, readback: bool = True):
        st = self._stream()
        ws = self.ws.data_ptr()
        g = self.scene.struct()
        for _ in range(4):
            abi.check(abi.unigs_preprocess(self.plan, g, self.cams, ws, st), "unigs_preprocess")
            if not readback:
                abi.check(abi.unigs_bin_sort(self.plan, ws, None, st), "unigs_bin_sort")
                return
            n = ctypes.c_int64(0)
            s = abi.unigs_bin_sort(self.plan, ws, n, st)
            if s == abi.UNIGS_ERR_CAPACITY:
                self._plan(int(n.value * 1.25) + 4096)
                ws = self.ws.data_ptr()
                continue
            abi.check(s, "unigs_bin_sort")
            self.last_instances = int(n.value)
            return
        raise RuntimeError("instance capacity could not be satisfied")

    def forward(self, out: Optional[Dict[str, torch.Tensor]] = None, readback: bool = True,
                normal_d: bool = True) -> Dict[str, torch.Tensor]:
        out = out if out is not None else self.alloc_outputs()
        self.preprocess_and_sort(readback)
        st = self._stream()
        g = self.scene.struct()
        abi.check(abi.unigs_render_fwd(self.plan, g, self.ws.data_ptr(), self._out_struct(out), st),
                  "unigs_render_fwd")
        if normal_d:
            abi.check(abi.unigs_depth_normal_fwd(self.plan, self.cams, _ptr(out["depth"]),
                                                 _ptr(out["normal_d"]), st),
                      "unigs_depth_normal_fwd")
        return out

    # -------------------------------------------------------------- backward
    def alloc_grads(self) -> Dict[str, torch.Tensor]:
        return {k: torch.empty(v.shape, dtype=torch.float32, device=self.device)
                for k, v in zip(("mean", "quat", "scale", "opacity", "kfac", "sh", "sem"),
                                self.scene.tensors())}

    def backward(self, out: Dict[str, torch.Tensor], grad_out: Dict[str, Optional[torch.Tensor]],
                 grads: Optional[Dict[str, torch.Tensor]] = None, accumulate: bool = False,
                 g_depth_buf: Optional[torch.Tensor] = None) -> Dict[str, torch.Tensor]:
        """Parameter gradients from upstream gradients of the flat outputs.

        grad_out keys: rgb, depth, normal_g, kmap, logits, normal_d (None =
        zero).  Must follow the forward that produced ``out`` on this renderer.
        """
        st = self._stream()
        grads = grads if grads is not None else self.alloc_grads()
        g_depth = grad_out.get("depth")
        g_nd = grad_out.get("normal_d")
        if g_nd is not None:
            if g_depth_buf is None:
                g_depth_buf = torch.empty(self.n_pixels, dtype=torch.float32, device=self.device)
            abi.check(abi.unigs_depth_normal_bwd(self.plan, self.cams, _ptr(out["depth"]),
                                                 _ptr(g_nd), _ptr(g_depth), _ptr(g_depth_buf), st),
                      "unigs_depth_normal_bwd")
            g_depth = g_depth_buf
        go = abi.unigs_grad_outputs()
        go.rgb, go.depth = _ptr(grad_out.get("rgb")), _ptr(g_depth)
        go.normal_g, go.kmap = _ptr(grad_out.get("normal_g")), _ptr(grad_out.get("kmap"))
        go.logits = _ptr(grad_out.get("logits")) if self.scene.n_sem else None
        pg = abi.unigs_param_grads()
        for k in ("mean", "quat", "scale", "opacity", "kfac", "sh", "sem"):
            setattr(pg, k, _ptr(grads[k]) if grads[k].numel() else None)
        pg.accumulate = 1 if accumulate else 0
        g = self.scene.struct()
        abi.check(abi.unigs_render_bwd(self.plan, g, self.cams, self.ws.data_ptr(),
                                       self._out_struct(out), go, pg, st), "unigs_render_bwd")
        return grads

    # ------------------------------------------------------------------ loss
    def alloc_loss_grads(self) -> Dict[str, torch.Tensor]:
        P = self.n_pixels
        f = lambda c: torch.empty(c * P, dtype=torch.float32, device=self.device)
        return {"rgb": f(3), "depth": f(1), "normal_d": f(3), "kmap": f(1),
                "logits": f(self.scene.n_sem)}

    def loss(self, out: Dict[str, torch.Tensor], targets: Dict[str, Optional[torch.Tensor]],
             record: torch.Tensor, lgrads: Dict[str, torch.Tensor], lam=None) -> torch.Tensor:
        """The combined loss of Sec. 3.4 (unigs_loss, include/unigs_train.h)
        on the outputs of the last forward: fills ``record`` (device float[16])
        and the gradients ``lgrads`` (rgb, depth, normal_d, kmap, logits),
        which :meth:`backward` takes as its upstream gradients."""
        t = abi.unigs_targets()
        t.rgb, t.depth = _ptr(targets.get("rgb")), _ptr(targets.get("depth"))
        t.normal = _ptr(targets.get("normal"))
        t.label = _ptr(targets.get("label")) if self.scene.n_sem else None
        g = abi.unigs_loss_grads()
        for k in ("rgb", "depth", "normal_d", "kmap", "logits"):
            x = lgrads.get(k)
            setattr(g, k, _ptr(x) if x is not None and x.numel() else None)
        if lam is None:
            lam = abi.unigs_loss_lambda_default()
        abi.check(abi.unigs_loss(self.plan, self._out_struct(out), _ptr(out["normal_d"]), t, lam,
                                 self.ws.data_ptr(), record.data_ptr(), g, self._stream()),
                  "unigs_loss")
        return record

    # ----------------------------------------------------------------- misc
    def status(self):
        d = ctypes.c_int64(0)
        s = abi.unigs_status_poll(self.plan, self.ws.data_ptr(), d, self._stream())
        return s, int(d.value)

    def stats(self):
        """(pairs evaluated, pairs blended) by the last forward."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        abi.check(abi.unigs_stats_poll(self.plan, self.ws.data_ptr(), a, b, self._stream()),
                  "unigs_stats_poll")
        return int(a.value), int(b.value)

    def launches_per_step(self) -> int:
        return abi.unigs_launches_per_step(self.plan)

    def sorted_instances(self):
        """(keys uint64, vals uint32, ranges [n_tiles,2] uint32) from the workspace."""
        s, _ = self.status()
        abi.check(s, "status")
        n = int(self.ws[self.plan.off[0] + 4: self.plan.off[0] + 8].view(torch.int32).item())
        fin = int(self.plan.sort_passes) & 1
        ko = self.plan.off[8 + fin]
        vo = self.plan.off[10 + fin]
        keys = self.ws[ko: ko + 8 * n].view(torch.int64).cpu().numpy().view(np.uint64)
        vals = self.ws[vo: vo + 4 * n].view(torch.int32).cpu().numpy().view(np.uint32)
        ro = self.plan.off[13]
        nt = int(self.plan.n_tiles)
        ranges = self.ws[ro: ro + 8 * nt].view(torch.int32).cpu().numpy().view(np.uint32)
        return keys, vals, ranges.reshape(nt, 2)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer: Renderer, mean, quat, scale, opacity, kfac, sh, sem):
        out = renderer.forward()
        ctx.renderer = renderer
        ctx.out = out
        return (out["rgb"], out["depth"], out["normal_g"], out["kmap"], out["logits"],
                out["normal_d"])

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_ng, g_k, g_log, g_nd):
        r: Renderer = ctx.renderer
        c = lambda x: None if x is None else x.contiguous()
        grads = r.backward(ctx.out, {"rgb": c(g_rgb), "depth": c(g_depth), "normal_g": c(g_ng),
                                     "kmap": c(g_k), "logits": c(g_log), "normal_d": c(g_nd)})
        sem_g = grads["sem"]
        sh_g = grads["sh"]
        return (None, grads["mean"], grads["quat"], grads["scale"], grads["opacity"],
                grads["kfac"], sh_g, sem_g)


def render(renderer: Renderer):
    """Differentiable render of ``renderer.scene``: returns flat (rgb, depth,
    normal_g, kmap, logits, normal_d); gradients flow to the scene tensors."""
    s = renderer.scene
    return _RenderFn.apply(renderer, s.mean, s.quat, s.scale, s.opacity, s.kfac, s.sh, s.sem)
