"""FP64 multimodal renderer of the oracle: the plain definition of the forward,
with its exact derivative taken by autograd.

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark use this module; the CUDA path never imports it.

What is computed (per camera, per pixel p = (u, v) at integer coordinates):

* Ray (Eq. computeRay, Sec. 3.2): origin C = t_cam^world, direction
  d = normalize(R_cam^world [(u-c_x)/f_x, (v-c_y)/f_y, 1]).
* Per Gaussian (Eq. 1): R from the normalised quaternion (w,x,y,z), S = diag(s).
  Local scaled ray (Sec. 3.2): v_l = R^T (C - mu), d_l = R^T d, v_s = v_l / s,
  d_s = d_l / s.  Quadratic of the supplement's Sec. 1:
  a = d_s.d_s, b = 2 v_s.d_s, c = v_s.v_s - 1.
* Depth (Eq. midpoint): t_mid = -b / 2a, d_i = t_mid * (R_world^cam d)_z, the
  camera-frame z of C + t_mid d.  t_mid is used for every ray, including rays
  that miss the 1-sigma ellipsoid (it is the Mahalanobis-closest point).
* Ray-ellipsoid normal of each Gaussian: the outward normal R S^-1 p of the
  ellipsoid at the scaled-space point p = v_s + t d_s, t the entry root
  (-b - sqrt(b^2-4ac)) / 2a; the exit root and a sign flip when the camera is
  inside the ellipsoid (c <= 0), so that n.d <= 0; the closest-approach point
  t_mid when the ray misses.  b^2 - 4ac is evaluated through the identity
  (b/2)^2 - ac = a - |v_s x d_s|^2.
* 2D splat (3DGS, which the paper extends, Sec. 3.4): centre m = (f_x x/z + c_x,
  f_y y/z + c_y) of p_c = R_wc mu + t_wc; covariance J W Sigma W^T J^T + 0.3 I
  with Sigma = R S S^T R^T; alpha = min(0.99, opacity * exp(-1/2 D^T conic D)),
  D = p - m.  A Gaussian is skipped where alpha < 1/255 or where the pixel
  lies outside its 3-sigma square |D_x| <= r, |D_y| <= r (r = ceil(3 sqrt of
  the larger eigenvalue of the 2D covariance), from the float32 binning
  recipe); the pixel stops before the first Gaussian that would bring T below
  1e-4.  (3DGS truncates to the tiles the square touches, which makes the
  image depend on the tile grid; the square itself does not.)
* Colour: max(0, SH(normalize(mu - C)) . h + 1/2).
* Compositing (Alg. 2 with T initialised to 1, Eqs. depth_render, t_render,
  semantic_render): w_i = alpha_i T_i; RGB, depth, normal, k and logits are
  sum_i w_i x_i over the tile list in front-to-back order; T_final is saved.
  Background is 0 in every channel.
* Normal from depth (Alg. 1 with the supplement's Sec. 3): back-project
  P_world = R_cw [x~ D, y~ D, D] + C, central differences at steps 1 and 2,
  n_g = v_x x v_y, n_2 aligned to n_1 (sign(0) = +1), fused with lambda = 0.5,
  normalised, then flipped if it points away from the camera.  A stencil
  reaching outside the image, or a zero fused vector, gives 0.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from .binning import project_fp32
from .sh import sh_basis

F64 = torch.float64
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
LOWPASS = 0.3


def _t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), dtype=F64)


@dataclasses.dataclass
class Params:
    """Gaussian parameters as float64 leaves (optionally requiring grad)."""
    mean: torch.Tensor     # [3,N]
    quat: torch.Tensor     # [4,N]
    scale: torch.Tensor    # [3,N]
    opacity: torch.Tensor  # [N]
    kfac: torch.Tensor     # [N]
    sh: torch.Tensor       # [N,n_sh,3]
    sem: torch.Tensor      # [N,C]
    sh_degree: int

    @staticmethod
    def from_scene(scene, requires_grad=False) -> "Params":
        ts = [_t(getattr(scene, k)) for k in
              ("mean", "quat", "scale", "opacity", "kfac", "sh", "sem")]
        for x in ts:
            x.requires_grad_(requires_grad)
        return Params(*ts, sh_degree=scene.sh_degree)

    def leaves(self):
        return [self.mean, self.quat, self.scale, self.opacity, self.kfac,
                self.sh, self.sem]


def quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    """[4,N] (w,x,y,z), any norm -> [N,3,3] rotation of the normalised quaternion."""
    q = q / torch.linalg.vector_norm(q, dim=0, keepdim=True)
    w, x, y, z = q
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


@dataclasses.dataclass
class Prep:
    """Per-(camera, Gaussian) float64 quantities feeding the composite."""
    mean2d: torch.Tensor   # [N,2]
    conic: torch.Tensor    # [N,3]  (A, B, C) of the inverse 2D covariance
    opacity: torch.Tensor  # [N]
    rgb: torch.Tensor      # [N,3]
    R: torch.Tensor        # [N,3,3]
    s: torch.Tensor        # [N,3]
    v_s: torch.Tensor      # [N,3]
    kfac: torch.Tensor     # [N]
    sem: torch.Tensor      # [N,C]
    z: torch.Tensor        # [N] camera-frame depth of the centre
    sh_raw: torch.Tensor   # [N,3] SH value + 1/2 before the clamp
    radius: torch.Tensor   # [N] 3-sigma radius r of the float32 recipe (pixels)

    def detached_leaves(self) -> "Prep":
        return Prep(*[x.detach().clone().requires_grad_(True)
                      for x in dataclasses.astuple(self)])

    def tensors(self):
        return [getattr(self, f.name) for f in dataclasses.fields(self)]


def preprocess(p: Params, cam) -> Prep:
    """Per-Gaussian projection, colour and ray-ellipsoid setup for one camera."""
    R_wc, t_wc, C = _t(cam.R_wc), _t(cam.t_wc), _t(cam.C)
    fx, fy, cx, cy = cam.fx, cam.fy, cam.cx, cam.cy
    mu = p.mean.T                                  # [N,3]
    pc = mu @ R_wc.T + t_wc                        # [N,3]
    x, y, z = pc.unbind(-1)
    R = quat_to_rot(p.quat)                        # [N,3,3]
    s = p.scale.T                                  # [N,3]
    M = R * s[:, None, :]                          # R S
    Sigma = M @ M.transpose(1, 2)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * x / (z * z)], -1),
                     torch.stack([zero, fy / z, -fy * y / (z * z)], -1)], -2)
    T = J @ R_wc                                   # [N,2,3]
    cov = T @ Sigma @ T.transpose(1, 2)
    ca = cov[:, 0, 0] + LOWPASS
    cb = cov[:, 0, 1]
    cc = cov[:, 1, 1] + LOWPASS
    det = ca * cc - cb * cb
    conic = torch.stack([cc / det, -cb / det, ca / det], -1)
    mean2d = torch.stack([fx * x / z + cx, fy * y / z + cy], -1)
    dirs = mu - C
    dirs = dirs / torch.linalg.vector_norm(dirs, dim=-1, keepdim=True)
    basis = sh_basis(dirs, p.sh_degree)            # [N,n_sh]
    sh_raw = torch.einsum("nk,nkc->nc", basis, p.sh) + 0.5
    rgb = torch.clamp(sh_raw, min=0.0)
    v_l = torch.einsum("nji,nj->ni", R, C - mu)    # R^T (C - mu)
    v_s = v_l / s
    return Prep(mean2d, conic, p.opacity, rgb, R, s, v_s, p.kfac, p.sem, z, sh_raw,
                recipe_radius(p, cam))


def recipe_radius(p: Params, cam) -> torch.Tensor:
    """The 3-sigma radius r of the float32 binning recipe (integer-valued) for
    the (float32-exact) parameters of ``p``; 0 where the recipe culls."""
    f32 = np.float32
    sc = dataclasses.make_dataclass("S", ["mean", "quat", "scale", "opacity"])(
        *[x.detach().numpy().astype(f32) for x in (p.mean, p.quat, p.scale, p.opacity)])
    pr = project_fp32(sc, cam)
    r = np.where(pr["valid"], pr["radius"], 0.0)
    return torch.as_tensor(r.astype(np.float64))


def pixel_rays(cam, uv: torch.Tensor):
    """Unit world ray directions d [P,3] and (R_wc d)_z [P] for pixel coords uv [P,2]."""
    R_cw, R_wc = _t(cam.R_cw), _t(cam.R_wc)
    dt = torch.stack([(uv[:, 0] - cam.cx) / cam.fx, (uv[:, 1] - cam.cy) / cam.fy,
                      torch.ones_like(uv[:, 0])], -1)
    d = dt @ R_cw.T
    d = d / torch.linalg.vector_norm(d, dim=-1, keepdim=True)
    zc = (d @ R_wc.T)[:, 2]
    return d, zc


def ray_ellipsoid(R: torch.Tensor, s: torch.Tensor, v_s: torch.Tensor,
                  d: torch.Tensor, zc: torch.Tensor, frozen=None):
    """Midpoint depth and ellipsoid normal for every (ray, Gaussian) pair.

    R [L,3,3], s [L,3], v_s [L,3] (= R^T (C - mu) / s), world ray directions
    d [P,3] (any length) and zc [P] = (R_wc d)_z.  Returns depth [P,L],
    normal [P,L,3] (world, unit, n.d <= 0), disc = (b^2-4ac)/4 [P,L], a [P,L]
    and c [L] of the quadratic of the supplement's Sec. 1.
    """
    d_l = torch.einsum("pj,ljk->plk", d, R)       # R^T d
    d_s = d_l / s[None]
    qa = (d_s * d_s).sum(-1)
    qb = 2.0 * (v_s[None] * d_s).sum(-1)
    qc = (v_s * v_s).sum(-1) - 1.0                 # [L]
    t_mid = -qb / (2.0 * qa)
    depth = t_mid * zc[:, None]

    cv = torch.cross(v_s[None].expand_as(d_s), d_s, dim=-1)
    disc = qa - (cv * cv).sum(-1)                  # (b^2 - 4ac) / 4
    with torch.no_grad():
        if frozen is not None and not isinstance(frozen, str):
            hit, inside = frozen
        else:
            hit = disc > 0
            inside = (qc <= 0)[None, :].expand_as(hit)
    sq = torch.sqrt(torch.where(hit, disc, torch.ones_like(disc))) * hit
    root_sign = torch.where(inside, torch.ones_like(disc), -torch.ones_like(disc))
    t_hit = (-0.5 * qb + root_sign * sq) / qa
    pnt = v_s[None] + t_hit[..., None] * d_s
    n_un = torch.einsum("lij,plj->pli", R, pnt / s[None])
    n = n_un / torch.linalg.vector_norm(n_un, dim=-1, keepdim=True)
    n = torch.where(inside[..., None], -n, n)
    if frozen is not None:
        return depth, n, disc, qa, qc, (hit, inside)
    return depth, n, disc, qa, qc


U32 = 2.0 ** -24          # unit roundoff of float32
EXP2_APPROX = 2.0 ** -21  # relative error allowed for the hardware exp2 approximation
SQUARE_BAND = 1e-4        # pixels: |D_x| or |D_y| this close to the 3-sigma radius
KAPPA_SPLIT = 65.0        # conic eigenvalue ratio above which the kernels evaluate the
                          # quadratic form in double-float (64, plus a margin for their
                          # float32 estimate of the ratio)


@dataclasses.dataclass
class Bands:
    """Widths of the bands around each discrete decision (test infrastructure:
    where a float64 decision lies inside its band, a float32 evaluation may
    decide the other way, so the pixel is not compared element-wise).

    ``alpha`` and ``T`` default to None: the width is then the first-order
    float32 error bound of the kernels' evaluation, per (pixel, Gaussian)
    pair for alpha and accumulated along the list for T (see
    :func:`alpha_error_bound`); a float gives a fixed relative width instead.
    ``inside`` bounds |c| = |v_s.v_s - 1| (camera inside the 1-sigma
    ellipsoid).  ``disc`` and ``disc_grad`` bound the relative discriminant
    delta = disc/a of the ray-ellipsoid quadratic: the kernels form
    disc = a - |v_s x d_s|^2 from float32 record entries, so near the
    silhouette (delta -> 0) disc carries an absolute error of about 4 u a.
    The normal moves like sqrt(disc), so its float32 error is about
    2 u / sqrt(delta): below 1e-4 for delta >= 1e-5 (``disc``).  Its
    derivative carries 1/sqrt(disc): a pair's gradient term is about
    delta^-1/2 times an ordinary one and off by 2 u / delta relative, i.e.
    2 u delta^-3/2 of an ordinary term, which stays below 1e-4 for
    delta >= 1e-2 (``disc_grad``).  ``clamp`` is a fixed width for alpha vs
    alpha_max when ``alpha`` is fixed."""
    alpha: Optional[float] = None
    T: Optional[float] = None
    inside: float = 1e-5
    disc: float = 1e-5
    clamp: float = 1e-5
    disc_grad: float = 1e-2


def alpha_error_bound(con: torch.Tensor, dx: torch.Tensor, dy: torch.Tensor,
                      kappa: torch.Tensor) -> torch.Tensor:
    """First-order relative error bound of a float32 evaluation of
    alpha = opacity * exp(-q/2), q = D^T K D, as the composite kernels do it.

    con [L,3] conic (A, B, C), dx, dy [P,L] pixel offsets, kappa [L] the
    conic's eigenvalue ratio.  With S = A dx^2 + C dy^2 + 2|B dx dy| (the sum
    of the absolute terms of q) and u = 2^-24:
      * float32 quadratic form (kappa <= KAPPA_SPLIT): rounding the conic to
        float32 and the three products and two additions give
        |dq| <= 4 u S (6 u S taken); otherwise the conditional form
        q = P w^2 + e b^2 with w = a + rho b formed from the exact offset by
        an error-free product and sum (rounded once) and P, e rounded to
        float32: each non-negative term carries 5 u (its inputs and two
        products) and the sum one more, |dq| <= 6 u q;
      * exp(-q/2) then carries a relative error q/2 * |dq|/q, plus q u from
        the rounded product x log2(e) inside the hardware exp, plus the exp2
        approximation (2^-21 taken);
      * the product with the opacity rounds once more (u).
    So beta = u (3 S + q + 1) + 2^-21 on the float32 path and
    u (4 q + 1) + 2^-21 on the conditional-form path."""
    q = con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy + 2.0 * con[None, :, 1] * dx * dy
    S = con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy \
        + 2.0 * (con[None, :, 1] * dx * dy).abs()
    f32_path = (kappa <= KAPPA_SPLIT)[None, :]
    beta32 = U32 * (3.0 * S + q + 1.0)
    betaff = U32 * (4.0 * q + 1.0)
    return torch.where(f32_path, beta32, betaff) + EXP2_APPROX


def conic_ratio(con: torch.Tensor) -> torch.Tensor:
    """Eigenvalue ratio lambda_max / lambda_min of the conics [L,3]."""
    a, b, c = con.unbind(-1)
    half = 0.5 * (a + c)
    rad = torch.sqrt(0.25 * (a - c) ** 2 + b * b)
    return (half + rad) / (half - rad)


def composite_tile(prep: Prep, ids: torch.Tensor, uv: torch.Tensor, cam,
                   bands: Optional[Bands] = None, frozen=None,
                   center_depth: bool = False) -> Dict[str, torch.Tensor]:
    """Alg. 2 for the pixels ``uv`` [P,2] over the ordered list ``ids`` [L].

    ``frozen`` (the ``decisions`` entry of an earlier call on the same pixels
    and list) replays that call's discrete decisions - alpha skip, stop,
    ray hit and camera-inside - so that the result is a smooth function of
    the parameters (used for finite differences of the almost-everywhere
    derivative).  ``center_depth`` blends the camera-frame depth of each
    Gaussian centre instead of the ray-ellipsoid midpoint (the centre-depth
    ablation of Tab. 6)."""
    P = uv.shape[0]
    L = ids.numel()
    C = prep.sem.shape[1]
    bands = bands or Bands()
    if L == 0:
        z = torch.zeros(P, dtype=F64)
        out = dict(rgb=torch.zeros(P, 3, dtype=F64), depth=z.clone(),
                   normal=torch.zeros(P, 3, dtype=F64), kmap=z.clone(),
                   logits=torch.zeros(P, C, dtype=F64), T=torch.ones(P, dtype=F64),
                   n_contrib=torch.zeros(P, dtype=torch.int64),
                   n_used=torch.zeros(P, dtype=torch.int64),
                   stats_eval=torch.zeros(P, dtype=torch.int64))
        for k in ("amb_fwd", "amb_grad"):
            out[k] = torch.zeros(P, dtype=torch.bool)
        out["decisions"] = None
        return out
    m = prep.mean2d[ids]
    con = prep.conic[ids]
    op = prep.opacity[ids]
    dx = uv[:, None, 0] - m[None, :, 0]
    dy = uv[:, None, 1] - m[None, :, 1]
    power = -0.5 * (con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) \
        - con[None, :, 1] * dx * dy
    a_raw = op[None, :] * torch.exp(power)
    alpha = torch.clamp(a_raw, max=ALPHA_MAX)
    rad = prep.radius[ids][None, :]
    with torch.no_grad():
        in_square = (dx.abs() <= rad) & (dy.abs() <= rad)
        valid = (alpha >= ALPHA_MIN) & in_square if frozen is None else frozen[0]
    a_eff = torch.where(valid, alpha, torch.zeros_like(alpha))
    one_m = 1.0 - a_eff
    T_after = torch.cumprod(one_m, dim=1)
    T_before = torch.cat([torch.ones(P, 1, dtype=F64), T_after[:, :-1]], dim=1)
    with torch.no_grad():
        incl = valid & (T_after >= T_MIN) if frozen is None else frozen[1]
    w = torch.where(incl, a_eff * T_before, torch.zeros_like(a_eff))
    T_final = torch.prod(torch.where(incl, one_m, torch.ones_like(one_m)), dim=1)

    # ray-ellipsoid intersection per (pixel, Gaussian)
    d, zc = pixel_rays(cam, uv)
    depth, n, disc, qa, qc, hit_inside = ray_ellipsoid(
        prep.R[ids], prep.s[ids], prep.v_s[ids], d, zc,
        frozen="return" if frozen is None else frozen[2])

    if center_depth:
        depth = prep.z[ids][None, :].expand_as(depth)
    rgb = w @ prep.rgb[ids]
    out = dict(
        rgb=rgb,
        depth=(w * depth).sum(1),
        normal=torch.einsum("pl,plc->pc", w, n),
        kmap=w @ prep.kfac[ids],
        logits=w @ prep.sem[ids],
        T=T_final,
    )
    out["decisions"] = (valid, incl, hit_inside)
    with torch.no_grad():
        pos = torch.arange(1, L + 1)[None, :].expand(P, L)
        out["n_contrib"] = torch.where(incl, pos, torch.zeros_like(pos)).max(1).values
        out["n_used"] = incl.sum(1)
        evaluated = T_before >= T_MIN
        # widths of the alpha and T bands: the float32 error bound of the
        # kernels' evaluation (Bands), or fixed relative widths
        if bands.alpha is None:
            beta = alpha_error_bound(con.detach(), dx.detach(), dy.detach(),
                                     conic_ratio(con.detach()))
        else:
            beta = torch.full_like(alpha, bands.alpha)
        clamp_w = beta if bands.alpha is None else torch.full_like(alpha, bands.clamp)
        if bands.T is None:
            # T after j blends: each blended alpha_j moves it by
            # alpha_j beta_j / (1 - alpha_j) (relative), and each product
            # 1 - alpha, T (1 - alpha) rounds twice
            ae = a_eff.detach()
            step = torch.where(valid, ae * beta / (1.0 - ae) + 2.0 * U32, torch.zeros_like(ae))
            beta_T = torch.cumsum(step, dim=1)
        else:
            beta_T = torch.full_like(alpha, bands.T)
        amb_alpha = (evaluated & in_square & ((alpha - ALPHA_MIN).abs() <= beta * alpha)).any(1)
        # the 3-sigma square: the kernels form |D| in float32 (error far below
        # 1e-4 px at these image sizes)
        near_edge = ((dx.abs() - rad).abs() <= SQUARE_BAND) | ((dy.abs() - rad).abs() <= SQUARE_BAND)
        amb_square = (evaluated & (alpha >= ALPHA_MIN) & near_edge).any(1)
        amb_T = (evaluated & valid & ((T_after - T_MIN).abs() <= beta_T * T_after)).any(1)
        amb_in = (incl & (qc.abs() <= bands.inside)[None, :]).any(1)
        rel_disc = disc / qa
        amb_disc = (incl & (rel_disc.abs() <= bands.disc)).any(1)
        amb_clamp = (incl & ((a_raw - ALPHA_MAX).abs() <= clamp_w * a_raw)).any(1)
        amb_dg = (incl & (rel_disc.abs() <= bands.disc_grad)).any(1)
        out["amb_fwd"] = amb_alpha | amb_T | amb_in | amb_disc | amb_square
        out["amb_grad"] = out["amb_fwd"] | amb_clamp | amb_dg
        out["stats_eval"] = evaluated.sum(1)
    return out


def tile_pixels(cam, tile_id_local: int, tile=(16, 16)):
    """Pixel coordinates (u, v) of a camera's tile (row-major tile ids, tiles
    of tile = (TW, TH) pixels)."""
    tw, th = (tile, tile) if isinstance(tile, int) else tile
    TX = (cam.width + tw - 1) // tw
    ty, tx = divmod(tile_id_local, TX)
    u = np.arange(tx * tw, min((tx + 1) * tw, cam.width))
    v = np.arange(ty * th, min((ty + 1) * th, cam.height))
    vv, uu = np.meshgrid(v, u, indexing="ij")
    return uu.ravel(), vv.ravel()


def render_camera(prep: Prep, cam, binning, cam_index: int,
                  tiles: Optional[Sequence[int]] = None,
                  bands: Optional[Bands] = None,
                  center_depth: bool = False) -> Dict[str, torch.Tensor]:
    """Composite every pixel of the listed local tiles (default: all) of one camera.

    Returns full-size planar images [C,H,W] (pixels of unlisted tiles are 0).
    """
    H, W = cam.height, cam.width
    tile = tuple(binning.get("tile", (16, 16)))
    TX = (W + tile[0] - 1) // tile[0]
    TY = (H + tile[1] - 1) // tile[1]
    C = prep.sem.shape[1]
    off = int(binning["tile_offset"][cam_index])
    ranges = binning["ranges"]
    vals = binning["vals"]
    outs = {k: torch.zeros(ch, H, W, dtype=F64) for k, ch in
            (("rgb", 3), ("depth", 1), ("normal", 3), ("kmap", 1), ("logits", C),
             ("T", 1))}
    ints = {k: torch.zeros(H, W, dtype=torch.int64) for k in ("n_contrib", "n_used", "stats_eval")}
    flags = {k: torch.zeros(H, W, dtype=torch.bool) for k in ("amb_fwd", "amb_grad")}
    tiles = range(TX * TY) if tiles is None else tiles
    for t in tiles:
        s0, s1 = ranges[off + t]
        ids = torch.as_tensor(vals[s0:s1].astype(np.int64))
        uu, vv = tile_pixels(cam, t, tile)
        uv = torch.as_tensor(np.stack([uu, vv], 1), dtype=F64)
        r = composite_tile(prep, ids, uv, cam, bands, center_depth=center_depth)
        vi = torch.as_tensor(vv)
        ui = torch.as_tensor(uu)
        for k in outs:
            val = r[k] if r[k].dim() == 2 else r[k][:, None]
            outs[k] = _put(outs[k], vi, ui, val)
        for k in ints:
            ints[k][vi, ui] = r[k]
        for k in flags:
            flags[k][vi, ui] = r[k]
    res = {k: (v[0] if v.shape[0] == 1 else v) for k, v in outs.items()}
    res.update(ints)
    res.update(flags)
    return res


def _put(img, vi, ui, val):
    """Functional scatter of val [P,C] into img [C,H,W] (keeps autograd)."""
    Cc, H, W = img.shape
    flat = img.reshape(Cc, H * W)
    idx = (vi * W + ui)
    flat = flat.index_copy(1, idx, val.T.contiguous())
    return flat.reshape(Cc, H, W)


def depth_to_normal(D: torch.Tensor, cam, step1: int = 1, step2: int = 2,
                    lam: float = 0.5) -> Dict[str, torch.Tensor]:
    """Alg. 1 on a float64 depth map D [H,W]; returns the normal [3,H,W] (world)."""
    H, W = D.shape
    R_cw, C = _t(cam.R_cw), _t(cam.C)
    v, u = torch.meshgrid(torch.arange(H, dtype=F64), torch.arange(W, dtype=F64),
                          indexing="ij")
    xt = (u - cam.cx) / cam.fx
    yt = (v - cam.cy) / cam.fy
    Pc = torch.stack([xt * D, yt * D, D])                      # [3,H,W]
    Pw = torch.einsum("ij,jhw->ihw", R_cw, Pc) + C[:, None, None]

    def normal_at(g):
        n = torch.zeros(3, H, W, dtype=F64)
        ok = torch.zeros(H, W, dtype=torch.bool)
        if H > 2 * g and W > 2 * g:
            vx = Pw[:, g:H - g, 2 * g:W] - Pw[:, g:H - g, 0:W - 2 * g]
            vy = Pw[:, 2 * g:H, g:W - g] - Pw[:, 0:H - 2 * g, g:W - g]
            nin = torch.cross(vx, vy, dim=0)
            n = torch.nn.functional.pad(nin, (g, g, g, g))
            ok[g:H - g, g:W - g] = True
        return n, ok

    n1, ok1 = normal_at(step1)
    n2, ok2 = normal_at(step2)
    dot12 = (n1 * n2).sum(0)
    with torch.no_grad():
        sgn = torch.where(dot12 >= 0, 1.0, -1.0).to(F64)
    nf = lam * n1 + (1.0 - lam) * n2 * sgn
    norm = torch.linalg.vector_norm(nf, dim=0)
    with torch.no_grad():
        ok = ok1 & ok2 & (norm > 0)
    N = nf / torch.where(ok, norm, torch.ones_like(norm))
    N = torch.where(ok[None], N, torch.zeros_like(N))
    dview = C[:, None, None] - Pw
    dn = (N * dview).sum(0)
    with torch.no_grad():
        flip = dn < 0
        # decision margins for the tests: n1.n2 near 0, N.d_view near 0
        n1n = torch.linalg.vector_norm(n1, dim=0)
        n2n = torch.linalg.vector_norm(n2, dim=0)
        amb = ok & (((dot12.abs() <= 1e-6 * n1n * n2n)) |
                    (dn.abs() <= 1e-6 * torch.linalg.vector_norm(dview, dim=0)) |
                    (norm <= 1e-9 * (n1n + n2n)))
    N = torch.where(flip[None], -N, N)
    return dict(normal=N, valid=ok, amb=amb)
