"""Seeded synthetic inputs: Gaussian scenes, cameras and upstream gradients.

This module only draws random numbers and builds camera poses.  It holds none
of the rasterizer's arithmetic, so both the CUDA path and the FP64 oracle can
take their inputs from it.

Every array is drawn in float64 with ``numpy.random.default_rng(seed)`` and
rounded once to the storage precision (float32, or bfloat16 for the feature
arrays of the BF16 configurations).  Both sides are fed the same rounded
values.

Scene shapes follow the paper's indoor workloads (Replica-like rooms with
50k-240k Gaussians, Tab. 4 and Tab. 6), scaled to the sizes of the benchmark
configurations:

* ``config1``: 10k Gaussians in a slab in front of one 256x256 camera.
* ``room``: points within 5 cm of the six walls of a 6x3x6 m room and of ten
  boxes standing on its floor, sampled in proportion to area.

World frame: +y points down (so a camera with identity rotation has x right,
y down, z forward, the camera frame of the back-projection in the supplement's
"Depth Backprojection" paragraph).  The floor is the plane y = +1.5.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

ROOM_HALF = np.array([3.0, 1.5, 3.0])


# ----------------------------------------------------------------------------
# bfloat16 rounding (round-to-nearest-even), used to make the BF16-stored
# feature arrays; the values are kept as float32 holding exact bf16 numbers.
# ----------------------------------------------------------------------------
def round_to_bf16(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of float32 values that are already bf16-exact."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return (u >> np.uint32(16)).astype(np.uint16)


# ----------------------------------------------------------------------------
# Cameras
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Camera:
    """Pinhole camera, rounded once from float64 to float32.

    ``R_wc``/``t_wc`` map world to camera (p_c = R_wc p + t_wc); ``R_cw`` and
    ``C`` are the camera-to-world rotation and the camera centre, the
    quantities the paper's ray equation uses.  All matrices are row-major.
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R_wc: np.ndarray  # (3,3) float32
    t_wc: np.ndarray  # (3,)  float32
    R_cw: np.ndarray  # (3,3) float32
    C: np.ndarray     # (3,)  float32
    z_near: float = 0.2

    @staticmethod
    def from_pose(width: int, height: int, f: float, R_cw64: np.ndarray,
                  C64: np.ndarray, z_near: float = 0.2) -> "Camera":
        R_cw64 = np.asarray(R_cw64, dtype=np.float64)
        C64 = np.asarray(C64, dtype=np.float64)
        R_wc64 = R_cw64.T
        t_wc64 = -R_wc64 @ C64
        f32 = np.float32
        return Camera(width=int(width), height=int(height),
                      fx=float(f32(f)), fy=float(f32(f)),
                      cx=float(f32(width / 2.0)), cy=float(f32(height / 2.0)),
                      R_wc=R_wc64.astype(np.float32),
                      t_wc=t_wc64.astype(np.float32),
                      R_cw=R_wc64.T.astype(np.float32),
                      C=C64.astype(np.float32),
                      z_near=float(f32(z_near)))


def look_at(C: Sequence[float], target: Sequence[float],
            up: Sequence[float] = (0.0, -1.0, 0.0)) -> np.ndarray:
    """Camera-to-world rotation whose columns are (right, down, forward)."""
    C = np.asarray(C, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - C
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, dtype=np.float64)
    down = -(up - fwd * np.dot(up, fwd))
    down /= np.linalg.norm(down)
    right = np.cross(down, fwd)
    return np.stack([right, down, fwd], axis=1)


def orbit_cameras(n: int, seed: int, resolutions: Sequence[tuple],
                  radius: float = 1.5) -> List[Camera]:
    """``n`` cameras on a horizontal circle looking at the room centre.

    Angles 2*pi*k/n + U(-0.1, 0.1), pitch U(-0.1, 0.1), focal 0.9375 * width
    (a 56 degree horizontal field of view).
    """
    rng = np.random.default_rng(seed)
    cams = []
    for k in range(n):
        ang = 2.0 * math.pi * k / n + rng.uniform(-0.1, 0.1)
        pitch = rng.uniform(-0.1, 0.1)
        C = np.array([radius * math.cos(ang), 0.0, radius * math.sin(ang)])
        target = np.array([0.0, math.tan(pitch) * radius, 0.0])
        w, h = resolutions[k % len(resolutions)] if len(resolutions) else (640, 480)
        cams.append(Camera.from_pose(w, h, 0.9375 * w, look_at(C, target), C))
    return cams


def front_camera(width: int, height: int, f: float) -> Camera:
    return Camera.from_pose(width, height, f, np.eye(3), np.zeros(3))


# ----------------------------------------------------------------------------
# Gaussian scenes
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Scene:
    """Gaussian parameters in the layout the library takes.

    mean [3][N], quat [4][N] (w,x,y,z, not normalised), scale [3][N] (>0),
    opacity [N] in (0,1), kfac [N], sh [N][n_sh][3], sem [N][n_sem].
    ``feat_bf16`` marks sh/sem as bf16-exact values (stored as bf16 on the
    device).
    """
    mean: np.ndarray
    quat: np.ndarray
    scale: np.ndarray
    opacity: np.ndarray
    kfac: np.ndarray
    sh: np.ndarray
    sem: np.ndarray
    sh_degree: int
    feat_bf16: bool = False

    @property
    def n(self) -> int:
        return self.mean.shape[1]

    @property
    def n_sem(self) -> int:
        return self.sem.shape[1]

    def subset(self, idx: np.ndarray) -> "Scene":
        return Scene(self.mean[:, idx].copy(), self.quat[:, idx].copy(),
                     self.scale[:, idx].copy(), self.opacity[idx].copy(),
                     self.kfac[idx].copy(), self.sh[idx].copy(),
                     self.sem[idx].copy(), self.sh_degree, self.feat_bf16)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _random_quats(rng, n):
    q = rng.normal(size=(4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    # leave them unnormalised by a random factor: the library normalises
    return q * rng.uniform(0.5, 2.0, size=(1, n))


def _room_surfaces(rng, n_boxes=10):
    """List of (origin, edge_u, edge_v, inward normal) rectangles."""
    hx, hy, hz = ROOM_HALF
    surf = []
    # six walls, normals pointing into the room
    surf.append(((-hx, -hy, -hz), (0, 2 * hy, 0), (0, 0, 2 * hz), (1, 0, 0)))
    surf.append(((hx, -hy, -hz), (0, 2 * hy, 0), (0, 0, 2 * hz), (-1, 0, 0)))
    surf.append(((-hx, -hy, -hz), (2 * hx, 0, 0), (0, 0, 2 * hz), (0, 1, 0)))
    surf.append(((-hx, hy, -hz), (2 * hx, 0, 0), (0, 0, 2 * hz), (0, -1, 0)))
    surf.append(((-hx, -hy, -hz), (2 * hx, 0, 0), (0, 2 * hy, 0), (0, 0, 1)))
    surf.append(((-hx, -hy, hz), (2 * hx, 0, 0), (0, 2 * hy, 0), (0, 0, -1)))
    for _ in range(n_boxes):
        sx, sy, sz = rng.uniform(0.2, 1.0, size=3)
        cx = rng.uniform(-hx + sx / 2, hx - sx / 2)
        cz = rng.uniform(-hz + sz / 2, hz - sz / 2)
        x0, x1 = cx - sx / 2, cx + sx / 2
        z0, z1 = cz - sz / 2, cz + sz / 2
        y1 = hy            # floor
        y0 = hy - sy       # box top (y points down)
        surf.append(((x0, y0, z0), (sx, 0, 0), (0, 0, sz), (0, -1, 0)))  # top
        surf.append(((x0, y0, z0), (0, sy, 0), (0, 0, sz), (-1, 0, 0)))
        surf.append(((x1, y0, z0), (0, sy, 0), (0, 0, sz), (1, 0, 0)))
        surf.append(((x0, y0, z0), (sx, 0, 0), (0, sy, 0), (0, 0, -1)))
        surf.append(((x0, y0, z1), (sx, 0, 0), (0, sy, 0), (0, 0, 1)))
        del y1
    return [tuple(np.asarray(a, dtype=np.float64) for a in s) for s in surf]


def _room_points(rng, n):
    surf = _room_surfaces(rng)
    areas = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v, _ in surf])
    which = rng.choice(len(surf), size=n, p=areas / areas.sum())
    a = rng.uniform(size=n)
    b = rng.uniform(size=n)
    off = rng.uniform(-0.05, 0.05, size=n)
    O = np.stack([s[0] for s in surf])[which]
    U = np.stack([s[1] for s in surf])[which]
    V = np.stack([s[2] for s in surf])[which]
    Nn = np.stack([s[3] for s in surf])[which]
    P = O + a[:, None] * U + b[:, None] * V + off[:, None] * Nn
    return P.T.copy()


def make_scene(kind: str, n: int, n_sem: int, sh_degree: int, seed: int,
               log_scale_mean: float = -4.0, log_scale_std: float = 0.5,
               log_scale_max: Optional[float] = None,
               feat_bf16: bool = False) -> Scene:
    """Draw a seeded scene.  ``kind`` is "slab" (config 1) or "room"."""
    rng = np.random.default_rng(seed)
    if kind == "slab":
        mean = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                         rng.uniform(2, 6, n)])
    elif kind == "room":
        mean = _room_points(rng, n)
    else:
        raise ValueError(kind)
    log_s = rng.normal(log_scale_mean, log_scale_std, size=(3, n))
    if log_scale_max is not None:
        log_s = np.minimum(log_s, log_scale_max)
    scale = np.exp(log_s)
    quat = _random_quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, n))
    kfac = _sigmoid(rng.normal(2.0, 1.0, n))
    n_sh = (sh_degree + 1) ** 2
    if kind == "slab":
        # colours U[0,1] through the DC band: c = Y00 * h0 + 0.5
        y00 = 0.5 / math.sqrt(math.pi)
        col = rng.uniform(0, 1, size=(n, 3))
        sh = np.zeros((n, n_sh, 3))
        sh[:, 0, :] = (col - 0.5) / y00
    else:
        sh = rng.normal(0.0, 0.2, size=(n, n_sh, 3))
    sem = rng.normal(0.0, 1.0, size=(n, n_sem))
    f32 = np.float32
    sh = sh.astype(f32)
    sem = sem.astype(f32)
    if feat_bf16:
        sh = round_to_bf16(sh)
        sem = round_to_bf16(sem)
    return Scene(mean.astype(f32), quat.astype(f32), scale.astype(f32),
                 opacity.astype(f32), kfac.astype(f32),
                 np.ascontiguousarray(sh), np.ascontiguousarray(sem),
                 sh_degree, feat_bf16)


def upstream_grads(cams: Sequence[Camera], n_sem: int, seed: int,
                   scale: float = 1.0) -> dict:
    """N(0,1) upstream gradients per output channel and pixel, per camera.

    Returns a dict of lists (one array per camera) for rgb[3,H,W], depth[H,W],
    normal_g[3,H,W], kmap[H,W], logits[n_sem,H,W] and normal_d[3,H,W].
    """
    rng = np.random.default_rng(seed)
    out = {k: [] for k in ("rgb", "depth", "normal_g", "kmap", "logits", "normal_d")}
    for c in cams:
        H, W = c.height, c.width
        for k, ch in (("rgb", 3), ("depth", 1), ("normal_g", 3), ("kmap", 1),
                      ("logits", n_sem), ("normal_d", 3)):
            g = (rng.normal(size=(ch, H, W)) * scale).astype(np.float32)
            out[k].append(g[0] if k in ("depth", "kmap") else g)
    return out


# ----------------------------------------------------------------------------
# Named workloads (the benchmark configurations)
# ----------------------------------------------------------------------------
def config1():
    """Forward only: 10k Gaussians, one 256x256 camera, f=256, 16 logits."""
    sc = make_scene("slab", 10_000, 16, 0, seed=0)
    return sc, [front_camera(256, 256, 256.0)]


def config2():
    """200k room Gaussians, SH deg 3, 32 logits, one 640x480 camera f=600."""
    sc = make_scene("room", 200_000, 32, 3, seed=1)
    return sc, [front_camera(640, 480, 600.0)]


def config3(n: int = 1_000_000, feat_bf16: bool = False):
    """1M room Gaussians, heavy-tailed scales, SH deg 3, 64 logits, 1280x720."""
    sc = make_scene("room", n, 64, 3, seed=2, log_scale_mean=-4.5,
                    log_scale_std=1.0, log_scale_max=-1.0, feat_bf16=feat_bf16)
    return sc, [front_camera(1280, 720, 1200.0)]


def config3_orbit(n_cams: int = 16, n: int = 1_000_000, feat_bf16: bool = False):
    """The config-3 scene seen by ``n_cams`` 1280x720 cameras on the orbit."""
    sc, _ = config3(n, feat_bf16)
    return sc, orbit_cameras(n_cams, seed=12, resolutions=[(1280, 720)])


def config4(n: int = 3_000_000):
    """3M room Gaussians, 16 orbit cameras of mixed resolution, BF16 features."""
    sc = make_scene("room", n, 64, 3, seed=3, log_scale_mean=-4.5,
                    log_scale_std=1.0, log_scale_max=-1.0, feat_bf16=True)
    rng = np.random.default_rng(13)
    res = [(640, 480), (1280, 720), (1920, 1080)]
    pick = [res[i] for i in rng.integers(0, 3, size=16)]
    return sc, orbit_cameras(16, seed=14, resolutions=pick)


def small_room(n: int = 8000, width: int = 100, height: int = 76, n_sem: int = 8,
               sh_degree: int = 3, seed: int = 7, n_cams: int = 1,
               feat_bf16: bool = False, log_scale_mean: float = -2.6):
    """A small room scene for parity tests: several tiles and a ragged tail."""
    sc = make_scene("room", n, n_sem, sh_degree, seed, log_scale_mean=log_scale_mean,
                    log_scale_std=0.5, feat_bf16=feat_bf16)
    if n_cams == 1:
        cams = [Camera.from_pose(width, height, 0.9375 * width, np.eye(3), np.zeros(3))]
    else:
        cams = orbit_cameras(n_cams, seed=seed + 100,
                             resolutions=[(width, height), (width + 28, height - 20)])
    return sc, cams


def config5(n: int = 6_000_000):
    """Training workload: 6M room Gaussians, 8 orbit cameras at 1920x1080,
    64 logits, BF16 features."""
    sc = make_scene("room", n, 64, 3, seed=4, log_scale_mean=-4.5,
                    log_scale_std=1.0, log_scale_max=-1.0, feat_bf16=True)
    return sc, orbit_cameras(8, seed=15, resolutions=[(1920, 1080)])


def perturb(scene: "Scene", seed: int, sigma_mean: float = 0.01,
            sigma_log_scale: float = 0.1) -> "Scene":
    """A copy of ``scene`` with jittered centres and scales (the scene whose
    renders serve as training targets)."""
    rng = np.random.default_rng(seed)
    f32 = np.float32
    mean = (scene.mean + rng.normal(0, sigma_mean, scene.mean.shape)).astype(f32)
    scale = (scene.scale * np.exp(rng.normal(0, sigma_log_scale, scene.scale.shape))).astype(f32)
    return dataclasses.replace(scene, mean=mean, scale=scale)


def synthetic_maps(cams: Sequence[Camera], n_sem: int, seed: int) -> dict:
    """Stand-ins for rendered maps, per camera: rgb U(0,1), depth U(1,4),
    unit normal_d (10% of pixels zero, as where the stencil leaves the image),
    kmap U(0.5,1.5), logits N(0, 4)."""
    rng = np.random.default_rng(seed)
    out = {k: [] for k in ("rgb", "depth", "normal_d", "kmap", "logits")}
    for c in cams:
        H, W = c.height, c.width
        out["rgb"].append(rng.uniform(0, 1, (3, H, W)).astype(np.float32))
        out["depth"].append(rng.uniform(1, 4, (H, W)).astype(np.float32))
        n = rng.normal(size=(3, H, W))
        n /= np.linalg.norm(n, axis=0)
        n[:, rng.uniform(size=(H, W)) < 0.1] = 0.0
        out["normal_d"].append(n.astype(np.float32))
        out["kmap"].append(rng.uniform(0.5, 1.5, (H, W)).astype(np.float32))
        out["logits"].append(rng.normal(0, 2, (n_sem, H, W)).astype(np.float32))
    return out


def synthetic_targets(cams: Sequence[Camera], n_sem: int, seed: int) -> dict:
    """Training targets, per camera: rgb U(0,1); depth U(1,4) with 15% of the
    pixels unmeasured (0); unit normals; labels uniform in [0, n_sem) with
    10% unlabelled (-1)."""
    rng = np.random.default_rng(seed)
    out = {k: [] for k in ("rgb", "depth", "normal", "label")}
    for c in cams:
        H, W = c.height, c.width
        out["rgb"].append(rng.uniform(0, 1, (3, H, W)).astype(np.float32))
        d = rng.uniform(1, 4, (H, W))
        d[rng.uniform(size=(H, W)) < 0.15] = 0.0
        out["depth"].append(d.astype(np.float32))
        n = rng.normal(size=(3, H, W))
        out["normal"].append((n / np.linalg.norm(n, axis=0)).astype(np.float32))
        lab = rng.integers(0, max(n_sem, 1), (H, W))
        lab[rng.uniform(size=(H, W)) < 0.1] = -1
        out["label"].append(lab.astype(np.int32))
    return out


def anchor_set(n: int = 1000, n_offsets: int = 10, n_sem: int = 24, seed: int = 11,
               feat_dim: int = 32, hidden: int = 32, opacity_bias: float = 1.0):
    """Seeded synthetic anchor set and MLP parameters (row-per-anchor arrays,
    float32): anchors in a box in front of the identity camera of
    ``small_room`` (x in [-1.5, 1.5], y in [-1, 1], z in [2, 5]), log-normal
    scales around 0.07, offsets N(0, 1) in units of the scale, features and
    base logits N(0, 1), base k in [0.8, 1.2]; MLP weights N(0, 1/F) and
    N(0, 2/H) (unit-variance pre-activations), biases N(0, 0.1), the opacity
    branch's output bias shifted by ``opacity_bias``.  Returns (arrays, mlps)
    with mlps[name] = {w1 [H,F], b1 [H], w2 [out,H], b2 [out]}."""
    rng = np.random.default_rng(seed)
    f32 = np.float32
    lo, hi = np.array([-1.5, -1.0, 2.0]), np.array([1.5, 1.0, 5.0])
    arrs = {
        "pos": rng.uniform(lo, hi, size=(n, 3)).astype(f32),
        "scale": np.exp(rng.normal(-2.6, 0.3, size=(n, 3))).astype(f32),
        "offsets": rng.normal(0.0, 1.0, size=(n, n_offsets, 3)).astype(f32),
        "feat": rng.normal(0.0, 1.0, size=(n, feat_dim)).astype(f32),
        "sem": rng.normal(0.0, 1.0, size=(n, n_sem)).astype(f32),
        "kfac": rng.uniform(0.8, 1.2, size=n).astype(f32),
    }
    outs = {"sem": n_sem, "k": 1, "opacity": n_offsets, "color": 3 * n_offsets,
            "cov": 7 * n_offsets}
    mlps = {}
    for name, out in outs.items():
        if out == 0:
            continue
        mlps[name] = {
            "w1": (rng.normal(0.0, 1.0, size=(hidden, feat_dim)) / np.sqrt(feat_dim)).astype(f32),
            "b1": rng.normal(0.0, 0.1, size=hidden).astype(f32),
            "w2": (rng.normal(0.0, 1.0, size=(out, hidden)) * np.sqrt(2.0 / hidden)).astype(f32),
            "b2": (rng.normal(0.0, 0.1, size=out) + (opacity_bias if name == "opacity" else 0.0))
            .astype(f32),
        }
    return arrs, mlps
