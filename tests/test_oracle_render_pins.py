"""End-to-end pins of the oracle's forward: one Gaussian rendered through
``oracle.render`` (preprocess, pixel rays, binning and the tile composite),
checked against closed forms and independent numerical methods.

A single Gaussian that a pixel blends gives w = alpha and T = 1 - alpha, so
every output channel divided by 1 - T is that Gaussian's own value at the
pixel: its midpoint depth (Sec. 3.2, Eq. midpoint), its ellipsoid normal and
its SH colour.  The cameras are posed (rotation and translation both differ
from the identity), so the world-to-camera map, the camera centre and the
camera-to-world ray map of Eq. computeRay all enter.  CPU only.
"""
import json
import math
import os

import numpy as np
import scipy.linalg
import torch

import oracle
from paper_2510_12174_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _camera(width, height, f, cx, cy, R_cw, C):
    """A camera from an exactly representable pose (no rounding anywhere)."""
    R_cw = np.asarray(R_cw, dtype=np.float32)
    C = np.asarray(C, dtype=np.float32)
    R_wc = np.ascontiguousarray(R_cw.T)
    t_wc = (-(R_wc.astype(np.float64) @ C.astype(np.float64))).astype(np.float32)
    return scenes.Camera(width=width, height=height, fx=f, fy=f, cx=cx, cy=cy, R_wc=R_wc,
                         t_wc=t_wc, R_cw=np.ascontiguousarray(R_cw), C=C)


def _one_gaussian(mu, quat, s, opacity, sh, n_sem=2):
    f32 = np.float32
    sh = np.asarray(sh, dtype=f32)
    deg = int(round(math.sqrt(sh.shape[0]))) - 1
    return scenes.Scene(mean=np.asarray(mu, f32).reshape(3, 1),
                        quat=np.asarray(quat, f32).reshape(4, 1),
                        scale=np.asarray(s, f32).reshape(3, 1),
                        opacity=np.asarray([opacity], f32), kfac=np.asarray([1.0], f32),
                        sh=sh[None].copy(), sem=np.ones((1, n_sem), f32), sh_degree=deg)


def _render(sc, cam):
    _, outs, _ = oracle.render(sc, [cam], with_normal_d=False)
    r = outs[0]
    return {k: (v.numpy() if torch.is_tensor(v) else v) for k, v in r.items()}


def test_rendered_depth_of_axis_aligned_gaussian_matches_closed_form():
    """Posed camera, Gaussian on its optical axis with its axes along the
    camera axes: depth / (1 - T) at integer pixels equals the closed-form
    midpoint depth z0 / (1 + s_z^2 (x~^2/s_x^2 + y~^2/s_y^2)) of the fixture."""
    with open(os.path.join(GOLDEN, "axis_aligned_render.json")) as fh:
        fx = json.load(fh)
    c = fx["camera"]
    cam = _camera(c["width"], c["height"], c["f"], c["cx"], c["cy"], c["R_cw"], c["C"])
    n_checked = 0
    for case in fx["cases"]:
        sc = _one_gaussian(case["mu"], fx["quat"], case["s"], fx["opacity"], np.zeros((1, 3)))
        r = _render(sc, cam)
        for p in case["pixels"]:
            u, v = p["u"], p["v"]
            cover = 1.0 - r["T"][v, u]
            assert cover > 1.0 / 255.0, (case["z0"], u, v)
            got = r["depth"][v, u] / cover
            assert abs(got - p["depth"]) < 1e-10 * p["depth"], (case["z0"], u, v, got, p["depth"])
            n_checked += 1
    assert n_checked == 48


def _rot_from_quat_expm(q):
    """Rotation of a quaternion (w, x, y, z) as the matrix exponential of its
    axis-angle form (independent of the oracle's quaternion formula)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q)
    vn = np.linalg.norm(q[1:])
    ang = 2.0 * math.atan2(vn, q[0])
    ax = q[1:] / vn
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return scipy.linalg.expm(ang * K)


def test_rendered_normal_and_depth_of_rotated_gaussian_match_bisection():
    """Posed orbit camera and a rotated, anisotropic Gaussian: normal / (1 - T)
    equals the normalised gradient of the implicit ellipsoid at the entry point
    found by bisection on |S^-1 R^T (C + t d - mu)| = 1 (Sec. 3.2), and
    depth / (1 - T) equals the camera-frame z of the point of the ray that
    minimises the Mahalanobis distance, found by golden-section search."""
    rng = np.random.default_rng(41)
    cam = scenes.orbit_cameras(1, seed=9, resolutions=[(80, 64)])[0]
    R_cw = cam.R_cw.astype(np.float64)
    R_wc = cam.R_wc.astype(np.float64)
    C = cam.C.astype(np.float64)
    n_checked = 0
    for trial in range(6):
        pc = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.2, 0.2), rng.uniform(2.0, 3.5)])
        mu = (C + R_cw @ pc).astype(np.float32)
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        ang = rng.uniform(0.3, 2.8)
        q = (np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])
             * rng.uniform(0.5, 2.0)).astype(np.float32)
        s = np.exp(rng.normal(-2.3, 0.4, 3)).astype(np.float32)
        sc = _one_gaussian(mu, q, s, 0.9, np.zeros((1, 3)))
        r = _render(sc, cam)
        R = _rot_from_quat_expm(q.astype(np.float64))
        m64 = mu.astype(np.float64)
        A = R @ np.diag(1.0 / s.astype(np.float64) ** 2) @ R.T
        pcm = R_wc @ (m64 - C)
        mx = cam.fx * pcm[0] / pcm[2] + cam.cx
        my = cam.fy * pcm[1] / pcm[2] + cam.cy
        for _ in range(6):
            u = int(round(mx)) + int(rng.integers(-2, 3))
            v = int(round(my)) + int(rng.integers(-2, 3))
            if not (0 <= u < cam.width and 0 <= v < cam.height):
                continue
            cover = 1.0 - r["T"][v, u]
            if cover <= 1.0 / 255.0:
                continue
            d = R_cw @ np.array([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0])

            def maha(t):
                e = C + t * d - m64
                return e @ A @ e

            lo, hi = 0.0, 50.0
            gr = (math.sqrt(5) - 1) / 2
            for _ in range(300):
                a = hi - gr * (hi - lo)
                b = lo + gr * (hi - lo)
                if maha(a) < maha(b):
                    hi = b
                else:
                    lo = a
            t_mid = 0.5 * (lo + hi)
            depth_ref = t_mid * (R_wc @ d)[2]
            got_depth = r["depth"][v, u] / cover
            assert abs(got_depth - depth_ref) < 1e-7 * depth_ref, (trial, u, v)
            if maha(t_mid) >= 1.0 - 1e-6:
                continue  # the ray misses the 1-sigma ellipsoid: no entry point
            lo, hi = 0.0, t_mid
            for _ in range(200):
                m = 0.5 * (lo + hi)
                if maha(m) > 1.0:
                    lo = m
                else:
                    hi = m
            x = C + 0.5 * (lo + hi) * d
            g = A @ (x - m64)
            n_ref = g / np.linalg.norm(g)
            got_n = r["normal"][:, v, u] / cover
            assert np.abs(got_n - n_ref).max() < 1e-8, (trial, u, v, got_n, n_ref)
            assert got_n @ d < 0
            n_checked += 1
    assert n_checked >= 15


def test_rendered_colour_of_degree1_sh_matches_closed_form():
    """SH degree 1 (Sec. 3.4: colour as in 3DGS, reading 3): with the DC band
    and the three band-1 coefficients, the rendered colour / (1 - T) equals
    max(0, 1/2 + Y00 h0 + c1 (dir_y h1 + dir_z h2 + dir_x h3)), c1 =
    sqrt(3 / 4 pi), Y00 = 1 / (2 sqrt(pi)), dir = (mu - C)/|mu - C| in the
    world frame (no Condon-Shortley phase); the third channel is driven below
    zero and must clamp to 0."""
    cam = _camera(96, 80, 128.0, 48.0, 40.0, [[0, 0, 1], [0, 1, 0], [-1, 0, 0]],
                  [0.5, -0.25, 1.0])
    R_cw = cam.R_cw.astype(np.float64)
    C = cam.C.astype(np.float64)
    pc = np.array([0.375, -0.25, 3.0])
    mu = C + R_cw @ pc                      # exact: dyadic
    h = np.array([[0.25, -0.5, -4.0],      # DC
                  [0.75, -0.25, 0.5],      # band 1: y
                  [-0.5, 0.625, 0.25],     # band 1: z
                  [0.5, 0.375, -1.0]])     # band 1: x
    sc = _one_gaussian(mu, [1, 0, 1, 0], [0.125, 0.125, 0.125], 0.875, h)
    r = _render(sc, cam)
    dirv = (mu - C) / np.linalg.norm(mu - C)
    y00 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    col = 0.5 + y00 * h[0] + c1 * (dirv[1] * h[1] + dirv[2] * h[2] + dirv[0] * h[3])
    col_ref = np.maximum(col, 0.0)
    assert col[2] < 0 and col_ref[2] == 0.0
    u = int(round(cam.cx + cam.fx * pc[0] / pc[2]))
    v = int(round(cam.cy + cam.fy * pc[1] / pc[2]))
    n_checked = 0
    for du, dv in ((0, 0), (1, 0), (0, -1), (-2, 1), (2, 2)):
        cover = 1.0 - r["T"][v + dv, u + du]
        assert cover > 0.05
        got = r["rgb"][:, v + dv, u + du] / cover
        assert np.abs(got - col_ref).max() < 1e-12, (got, col_ref)
        n_checked += 1
    assert n_checked == 5
