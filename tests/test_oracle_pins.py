"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
independent numerical methods (quadrature, golden-section search, bisection,
matrix exponential, finite differences), brute force over all Gaussians and
invariants of the compositing equations.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
from oracle import binning as ob
from oracle import raster as orr
from oracle.sh import sh_basis
from paper_2510_12174_gb300 import scenes

F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- SH basis
def test_sh_basis_orthonormal():
    """Real SH to degree 3 are orthonormal on the sphere (Gauss-Legendre x
    uniform-phi quadrature, exact for these polynomial degrees)."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = sh_basis(torch.as_tensor(dirs), 3).numpy()
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_band_l1_is_linear_in_direction():
    d = torch.tensor([[0.6, 0.0, 0.8]], dtype=F64)
    Y = sh_basis(d, 1)[0].numpy()
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y, [0.5 / math.sqrt(math.pi), 0.0, c1 * 0.8, c1 * 0.6], atol=1e-15)


# ------------------------------------------------------------- quaternions
def test_quaternion_matches_matrix_exponential():
    rng = np.random.default_rng(0)
    for _ in range(20):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        ang = rng.uniform(-np.pi, np.pi)
        q = np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * axis]) * rng.uniform(0.3, 3)
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        R_ref = scipy.linalg.expm(ang * K)
        R = orr.quat_to_rot(torch.as_tensor(q[:, None]))[0].numpy()
        assert np.abs(R - R_ref).max() < 1e-12


# ------------------------------------------------- ray-ellipsoid: depth
def _single(mu, R, s, C=(0.0, 0.0, 0.0)):
    mu = np.asarray(mu, float)
    R = np.asarray(R, float)
    s = np.asarray(s, float)
    v_s = (R.T @ (np.asarray(C, float) - mu)) / s
    return (torch.as_tensor(R[None]), torch.as_tensor(s[None]), torch.as_tensor(v_s[None]))


def _rand_rot(rng):
    q = rng.normal(size=4)
    return orr.quat_to_rot(torch.as_tensor(q[:, None]))[0].numpy()


def test_depth_centre_ray_equals_centre_depth_any_shape():
    """A ray through the centre gives t_mid at the centre: depth = z of mu."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        mu = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(2, 8)])
        R = _rand_rot(rng)
        s = np.exp(rng.normal(-3, 1, 3))
        d = torch.as_tensor((mu / np.linalg.norm(mu))[None])
        zc = d[:, 2].clone()
        depth, *_ = orr.ray_ellipsoid(*_single(mu, R, s), d, zc)
        assert abs(depth.item() - mu[2]) < 1e-12 * mu[2]


def test_depth_axis_aligned_closed_form():
    """Axis-aligned ellipsoid on the optical axis: the Mahalanobis-closest
    point along the ray (x~, y~, 1) has depth z0 / (1 + s_z^2 (x~^2/s_x^2 + y~^2/s_y^2))."""
    with open(os.path.join(GOLDEN, "axis_aligned_depth.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        s = np.array(c["s"])
        dt = np.array([c["xt"], c["yt"], 1.0])
        d = torch.as_tensor(dt[None])
        depth, *_ = orr.ray_ellipsoid(*_single([0, 0, c["z0"]], np.eye(3), s), d,
                                      torch.tensor([1.0], dtype=F64))
        assert abs(depth.item() - c["depth"]) < 1e-12 * c["depth"]


def test_depth_rotated_matches_golden_section_minimum():
    """t_mid = argmin_t (r(t)-mu)^T Sigma^-1 (r(t)-mu), found by golden section."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        mu = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(2, 5)])
        R = _rand_rot(rng)
        s = np.exp(rng.normal(-2, 0.7, 3))
        Sinv = R @ np.diag(1 / s ** 2) @ R.T
        dt = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 1.0])

        def f(t):
            e = t * dt - mu
            return e @ Sinv @ e

        lo, hi = 0.0, 20.0
        g = (math.sqrt(5) - 1) / 2
        for _ in range(200):
            a = hi - g * (hi - lo)
            b = lo + g * (hi - lo)
            if f(a) < f(b):
                hi = b
            else:
                lo = a
        t_star = 0.5 * (lo + hi)
        depth, *_ = orr.ray_ellipsoid(*_single(mu, R, s), torch.as_tensor(dt[None]),
                                      torch.tensor([1.0], dtype=F64))
        assert abs(depth.item() - t_star) < 1e-7 * t_star


def test_depth_invariant_to_ray_direction_scale():
    rng = np.random.default_rng(3)
    mu = np.array([0.2, -0.1, 3.0])
    R = _rand_rot(rng)
    s = np.array([0.05, 0.2, 0.01])
    dt = np.array([0.05, 0.02, 1.0])
    d1 = torch.as_tensor(dt[None])
    d2 = d1 * 7.3
    a, *_ = orr.ray_ellipsoid(*_single(mu, R, s), d1, d1[:, 2].clone())
    b, *_ = orr.ray_ellipsoid(*_single(mu, R, s), d2, d2[:, 2].clone())
    assert abs(a.item() - b.item()) < 1e-13 * abs(a.item())


# ------------------------------------------------ ray-ellipsoid: normal
def test_normal_sphere_entry_point():
    """Sphere: the entry normal is (p - mu)/r at the geometric entry point."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        r = rng.uniform(0.05, 0.5)
        mu = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(2, 4)])
        # a ray through a point within the sphere's silhouette
        target = mu + rng.uniform(-0.6, 0.6, 3) * r
        d = target / np.linalg.norm(target)
        tc = d @ mu
        perp2 = mu @ mu - tc ** 2
        t_in = tc - math.sqrt(r * r - perp2)
        p = t_in * d
        n_ref = (p - mu) / r
        _, n, disc, *_ = orr.ray_ellipsoid(*_single(mu, _rand_rot(rng), [r, r, r]),
                                           torch.as_tensor(d[None]), torch.tensor([d[2]]))
        assert disc.item() > 0
        assert np.abs(n[0, 0].numpy() - n_ref).max() < 1e-10


def test_normal_rotated_ellipsoid_bisection():
    """Rotated ellipsoid: entry point by bisection on the implicit function
    |S^-1 R^T (x - mu)|^2 = 1 (Sec. 3.2), normal = its normalised gradient."""
    rng = np.random.default_rng(5)
    done = 0
    while done < 15:
        mu = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(2, 4)])
        R = _rand_rot(rng)
        s = np.exp(rng.normal(-2, 0.6, 3))
        A = R @ np.diag(1 / s ** 2) @ R.T
        d = (mu + rng.normal(size=3) * s.max() * 0.5)
        d /= np.linalg.norm(d)

        def f(t):
            e = t * d - mu
            return e @ A @ e - 1

        t_mid = (d @ A @ mu) / (d @ A @ d)
        if f(t_mid) >= 0:
            continue
        lo, hi = 0.0, t_mid
        for _ in range(200):
            m = 0.5 * (lo + hi)
            if f(m) > 0:
                lo = m
            else:
                hi = m
        x = 0.5 * (lo + hi) * d
        g = A @ (x - mu)
        n_ref = g / np.linalg.norm(g)
        _, n, *_ = orr.ray_ellipsoid(*_single(mu, R, s), torch.as_tensor(d[None]),
                                     torch.tensor([d[2]]))
        assert np.abs(n[0, 0].numpy() - n_ref).max() < 1e-8
        assert n[0, 0].numpy() @ d < 0
        done += 1


def test_normal_miss_is_perpendicular_and_inside_faces_camera():
    rng = np.random.default_rng(6)
    mu = np.array([0.0, 0.0, 3.0])
    R = _rand_rot(rng)
    s = np.array([0.1, 0.05, 0.02])
    d = np.array([0.3, 0.3, 1.0])
    d /= np.linalg.norm(d)  # far outside the ellipsoid: a miss
    _, n, disc, *_ = orr.ray_ellipsoid(*_single(mu, R, s), torch.as_tensor(d[None]),
                                       torch.tensor([d[2]]))
    assert disc.item() < 0
    assert abs(n[0, 0].numpy() @ d) < 1e-12
    # camera inside the ellipsoid: exit normal, flipped to face the camera
    mu = np.array([0.0, 0.0, 0.01])
    s = np.array([0.5, 0.4, 0.3])
    d = np.array([0.1, -0.2, 1.0])
    d /= np.linalg.norm(d)
    _, n, disc, qa, qc = orr.ray_ellipsoid(*_single(mu, R, s), torch.as_tensor(d[None]),
                                           torch.tensor([d[2]]))
    assert qc.item() < 0 and disc.item() > 0
    A = R @ np.diag(1 / s ** 2) @ R.T
    t_exit = (d @ A @ mu + math.sqrt((d @ A @ mu) ** 2 - (d @ A @ d) * (mu @ A @ mu - 1))) / (d @ A @ d)
    g = A @ (t_exit * d - mu)
    assert np.abs(n[0, 0].numpy() + g / np.linalg.norm(g)).max() < 1e-10
    assert n[0, 0].numpy() @ d < 0


def test_discriminant_identity_matches_paper_form():
    """(b^2 - 4ac)/4 of the supplement's quadratic equals a - |v_s x d_s|^2."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        v = rng.normal(size=3) * 3
        d = rng.normal(size=3)
        a, b, c = d @ d, 2 * v @ d, v @ v - 1
        R, s = np.eye(3), np.ones(3)
        _, _, disc, *_ = orr.ray_ellipsoid(torch.as_tensor(R[None]), torch.as_tensor(s[None]),
                                           torch.as_tensor(v[None]), torch.as_tensor(d[None]),
                                           torch.tensor([1.0], dtype=F64))
        assert abs(disc.item() - (b * b - 4 * a * c) / 4) < 1e-12 * (b * b + abs(4 * a * c))


# ------------------------------------------------------- projection pins
def test_projection_jacobian_is_derivative_of_pinhole():
    """The EWA Jacobian J is the derivative of (f_x x/z + c_x, f_y y/z + c_y):
    the oracle's 2D covariance equals J_fd W Sigma W^T J_fd^T + 0.3 I with J
    from central differences of the projection."""
    sc, cams = scenes.small_room(n=50, seed=11)
    cam = scenes.orbit_cameras(1, seed=3, resolutions=[(120, 90)])[0]
    p = orr.Params.from_scene(sc)
    pr = orr.preprocess(p, cam)
    R_wc = cam.R_wc.astype(np.float64)
    t_wc = cam.t_wc.astype(np.float64)
    for g in range(10):
        mu = sc.mean[:, g].astype(np.float64)
        pc = R_wc @ mu + t_wc
        if pc[2] < 0.5:
            continue

        def proj(x):
            return np.array([cam.fx * x[0] / x[2] + cam.cx, cam.fy * x[1] / x[2] + cam.cy])

        J = np.zeros((2, 3))
        h = 1e-6
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            J[:, k] = (proj(pc + e) - proj(pc - e)) / (2 * h)
        R = orr.quat_to_rot(torch.as_tensor(sc.quat[:, g:g + 1].astype(np.float64)))[0].numpy()
        S = np.diag(sc.scale[:, g].astype(np.float64))
        Sig = R @ S @ S @ R.T
        cov = J @ R_wc @ Sig @ R_wc.T @ J.T + 0.3 * np.eye(2)
        conic = np.linalg.inv(cov)
        got = pr.conic[g].numpy()
        assert np.allclose(got, [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6)
        assert np.allclose(pr.mean2d[g].numpy(), proj(pc), rtol=1e-13)


def test_fp32_recipe_tracks_fp64_projection():
    """The float32 binning recipe agrees with the float64 projection to float32
    rounding, and its radius covers the 3-sigma ellipse."""
    sc, cams = scenes.small_room(n=3000)
    cam = scenes.orbit_cameras(1, seed=5, resolutions=[(160, 120)])[0]
    pr32 = ob.project_fp32(sc, cam)
    pr64 = orr.preprocess(orr.Params.from_scene(sc), cam)
    v = pr32["valid"]
    assert v.sum() > 100
    m64 = pr64.mean2d.numpy()[v]
    assert np.abs(pr32["mean2d"].T[v] - m64).max() < 1e-5 * max(1.0, np.abs(m64).max())
    con = pr64.conic.numpy()[v]
    # 2D covariance from the float64 conic
    det = con[:, 0] * con[:, 2] - con[:, 1] ** 2
    cov = np.stack([con[:, 2] / det, -con[:, 1] / det, con[:, 0] / det], 1)
    rel = np.abs(pr32["cov2d"].T[v] - cov) / np.abs(cov).max(1, keepdims=True)
    assert rel.max() < 1e-5
    # 3-sigma extent along x and y is inside the radius
    r = pr32["radius"][v]
    assert np.all(3 * np.sqrt(cov[:, 0]) <= r + 1e-6)
    assert np.all(3 * np.sqrt(cov[:, 2]) <= r + 1e-6)


def _keep_scalar(pr, g, tx, ty, tile=(16, 16)):
    """The opacity-aware tile test written out with float32 scalars."""
    f = np.float32
    if pr["no_cull"][g]:
        return True
    mx, my = f(pr["mean2d"][0][g]), f(pr["mean2d"][1][g])
    kA, kB, kC = (f(pr["conic32"][i][g]) for i in range(3))
    tw, th = tile
    X0, X1, Y0, Y1 = f(tw * tx), f(tw * tx + tw - 1), f(th * ty), f(th * ty + th - 1)
    if X0 <= mx <= X1 and Y0 <= my <= Y1:
        return bool(f(0) <= pr["qlim"][g])
    best = None
    for xe in (X0, X1):
        dx = f(xe - mx)
        dy = min(max(f(f(-(f(kB * dx))) / kC), f(Y0 - my)), f(Y1 - my))
        q = f(f(f(f(kA * dx) * dx) + f(f(f(f(2) * kB) * dx) * dy)) + f(f(kC * dy) * dy))
        best = q if best is None else min(best, q)
    for ye in (Y0, Y1):
        dy = f(ye - my)
        dx = min(max(f(f(-(f(kB * dy))) / kA), f(X0 - mx)), f(X1 - mx))
        q = f(f(f(f(kA * dx) * dx) + f(f(f(f(2) * kB) * dx) * dy)) + f(f(kC * dy) * dy))
        best = min(best, q)
    return bool(best <= pr["qlim"][g])


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8), (64, 4)])
def test_binning_matches_brute_force_rect_enumeration(tile):
    sc, cams = scenes.small_room(n=600, n_cams=2, seed=9)
    b1 = ob.bin_cameras(sc, cams, tile)
    b2 = ob.bin_cameras_fast(sc, cams, tile)
    assert np.array_equal(b1["keys"], b2["keys"]) and np.array_equal(b1["vals"], b2["vals"])
    assert np.array_equal(b1["ranges"], b2["ranges"])
    # brute force: per tile, every Gaussian whose rectangle contains it and that
    # passes the tile test, ordered by (depth bits, index)
    n_culled = 0
    for k, cam in enumerate(cams):
        pr = b1["projs"][k]
        TX, TY = pr["tiles_x"], pr["tiles_y"]
        assert (TX, TY) == (-(-cam.width // tile[0]), -(-cam.height // tile[1]))
        x0, x1, y0, y1 = pr["rect"]
        # the rectangle covers the 3-sigma square [m - r, m + r] of every
        # valid Gaussian, in tiles of the requested shape
        v = pr["valid"]
        m, r = pr["mean2d"], pr["radius"]
        lo_x = np.clip(np.floor((m[0] - r) / tile[0]), 0, TX)
        hi_x = np.clip(np.ceil((m[0] + r) / tile[0]), 0, TX)
        assert np.array_equal(x0[v], lo_x[v]) and np.array_equal(x1[v], hi_x[v])
        lo_y = np.clip(np.floor((m[1] - r) / tile[1]), 0, TY)
        hi_y = np.clip(np.ceil((m[1] + r) / tile[1]), 0, TY)
        assert np.array_equal(y0[v], lo_y[v]) and np.array_equal(y1[v], hi_y[v])
        for t in range(TX * TY):
            ty, tx = divmod(t, TX)
            inside = pr["valid"] & (x0 <= tx) & (tx < x1) & (y0 <= ty) & (ty < y1)
            ids = [g for g in np.nonzero(inside)[0] if _keep_scalar(pr, g, tx, ty, tile)]
            n_culled += int(inside.sum()) - len(ids)
            ids = np.array(ids, dtype=np.int64)
            ids = ids[np.lexsort((ids, pr["zbits"][ids]))] if ids.size else ids
            s0, s1 = b1["ranges"][b1["tile_offset"][k] + t]
            assert np.array_equal(b1["vals"][s0:s1], ids)
    assert n_culled > 0


def test_render_does_not_depend_on_tile_shape():
    """The tile shape decides which (tile, Gaussian) pairs are listed, but the
    opacity-aware test drops only pairs whose alpha stays below 1/255 on the
    whole tile, and every tile's list is ordered by (depth, index): each pixel
    blends the same Gaussians in the same order for every shape."""
    sc, cams = scenes.small_room(n=3000, width=70, height=52, n_sem=4, seed=19, n_cams=2)
    ref = None
    for tile in ((16, 16), (8, 32), (32, 8), (64, 4)):
        _, outs, b = oracle.render(sc, cams, with_normal_d=False, tile=tile)
        assert b["tile"] == tile
        if ref is None:
            ref = outs
            continue
        for o, o0 in zip(outs, ref):
            for key in ("rgb", "depth", "normal", "kmap", "logits", "T"):
                assert torch.allclose(o[key], o0[key], rtol=1e-12, atol=1e-13), (tile, key)
            assert torch.equal(o["n_used"], o0["n_used"])


def test_tile_culling_is_conservative():
    """Every (tile, Gaussian) pair the opacity-aware test drops has float64
    alpha < 1/255 at every pixel of the tile (so Alg. 2 would skip it)."""
    sc, cams = scenes.small_room(n=4000, width=90, height=70, seed=19)
    cam = cams[0]
    pr = ob.project_fp32(sc, cam)
    prep = orr.preprocess(orr.Params.from_scene(sc), cam)
    idx = np.nonzero(pr["valid"])[0]
    gg, tx, ty = ob._rect_tiles(pr, idx)
    keep = ob.tile_keep(pr, gg, tx, ty)
    drop = np.nonzero(~keep)[0]
    assert 0.3 < drop.size / keep.size
    m = prep.mean2d.detach().numpy()
    con = prep.conic.detach().numpy()
    op = sc.opacity.astype(np.float64)
    worst = 0.0
    for j in drop:
        g = gg[j]
        u = np.arange(16 * tx[j], 16 * tx[j] + 16)
        v = np.arange(16 * ty[j], 16 * ty[j] + 16)
        vv, uu = np.meshgrid(v, u, indexing="ij")
        dx, dy = uu - m[g, 0], vv - m[g, 1]
        q = con[g, 0] * dx * dx + 2 * con[g, 1] * dx * dy + con[g, 2] * dy * dy
        worst = max(worst, float((op[g] * np.exp(-0.5 * q)).max() * 255.0))
    assert worst < 1.0


# -------------------------------------------------------- compositing
def _brute_force_pixel(prep, binproj, cam, u, v, ids_all):
    """Alg. 2 for one pixel, sequentially, over every Gaussian the recipe keeps
    whose 3-sigma square |u - m_x| <= r, |v - m_y| <= r contains the pixel -
    no tiles involved - ordered by (depth bits, index)."""
    m64 = prep.mean2d.numpy()
    r = binproj["radius"]
    sel = [g for g in ids_all if binproj["valid"][g] and abs(u - m64[g, 0]) <= r[g]
           and abs(v - m64[g, 1]) <= r[g]]
    sel.sort(key=lambda g: (int(binproj["zbits"][g]), g))
    d, zc = orr.pixel_rays(cam, torch.tensor([[float(u), float(v)]], dtype=F64))
    T = 1.0
    acc = np.zeros(3 + 1 + 3 + 1 + prep.sem.shape[1])
    for g in sel:
        m = prep.mean2d[g].numpy()
        A, B, Cc = prep.conic[g].numpy()
        dx, dy = u - m[0], v - m[1]
        alpha = min(0.99, prep.opacity[g].item() * math.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy))
        if alpha < 1 / 255:
            continue
        if T * (1 - alpha) < 1e-4:
            break
        depth, n, *_ = orr.ray_ellipsoid(prep.R[g:g + 1], prep.s[g:g + 1], prep.v_s[g:g + 1], d, zc)
        feat = np.concatenate([prep.rgb[g].numpy(), [depth.item()], n[0, 0].numpy(),
                               [prep.kfac[g].item()], prep.sem[g].numpy()])
        acc += alpha * T * feat
        T *= 1 - alpha
    return acc, T


def test_composite_matches_brute_force_per_pixel():
    sc, cams = scenes.small_room(n=6000, width=40, height=36, n_sem=4, log_scale_mean=-2.3)
    cam = cams[0]
    _, outs, b = oracle.render(sc, cams, with_normal_d=False)
    r = outs[0]
    prep = orr.preprocess(orr.Params.from_scene(sc), cam)
    rng = np.random.default_rng(0)
    ids_all = list(range(sc.n))
    pix = [(rng.integers(0, 40), rng.integers(0, 36)) for _ in range(25)]
    checked_term = 0
    for u, v in pix:
        acc, T = _brute_force_pixel(prep, b["projs"][0], cam, int(u), int(v), ids_all)
        got = np.concatenate([r["rgb"][:, v, u].numpy(), [r["depth"][v, u].item()],
                              r["normal"][:, v, u].numpy(), [r["kmap"][v, u].item()],
                              r["logits"][:, v, u].numpy()])
        assert np.abs(got - acc).max() < 1e-12
        assert abs(r["T"][v, u].item() - T) < 1e-12
        checked_term += T < 1e-3
    assert checked_term > 0  # some sampled pixels reached the termination rule


def test_composite_invariants():
    """T_final + sum w = 1; unit features render 1 - T_final; all k = 1 gives
    K = 1 - T_final (the supplement's analysis of k = 1); linearity in o."""
    sc, cams = scenes.small_room(n=6000, width=48, height=40, n_sem=3, log_scale_mean=-2.3)
    sc.kfac[:] = 1.0
    sc.sem[:, 0] = 1.0
    sc.sh[:] = 0.0
    sc.sh[:, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))  # colour exactly 1
    _, outs, _ = oracle.render(sc, cams, with_normal_d=False)
    r = outs[0]
    one_minus_T = 1 - r["T"]
    assert (r["T"] < 1e-3).float().mean() > 0.02
    assert torch.abs(r["kmap"] - one_minus_T).max() < 1e-12
    assert torch.abs(r["logits"][0] - one_minus_T).max() < 1e-12
    col = 0.5 / math.sqrt(math.pi) * float(sc.sh[0, 0, 0]) + 0.5   # 1 up to float32 rounding
    assert torch.abs(r["rgb"] - col * one_minus_T[None]).max() < 1e-12
    sc2 = scenes.Scene(**{**sc.__dict__})
    sc2.sem = sc.sem.astype(np.float64) * 2.5
    _, outs2, _ = oracle.render(sc2, cams, with_normal_d=False)
    assert torch.abs(outs2[0]["logits"] - 2.5 * r["logits"]).max() < 1e-12


def test_center_depth_ablation_blends_centre_z():
    """Centre-depth mode (Tab. 6 ablation): D = sum_i w_i z_i with z_i the
    camera-frame depth of the centre and the weights of Alg. 2.  Pinned through
    the K channel: with k_i := z_i, Eq. t_render gives the same sum."""
    sc, cams = scenes.small_room(n=3000, width=40, height=32, n_sem=2, seed=23)
    cam = cams[0]
    _, a, b = oracle.render(sc, cams, with_normal_d=False)
    _, c, _ = oracle.render(sc, cams, with_normal_d=False, binning=b, center_depth=True)
    assert torch.equal(a[0]["rgb"], c[0]["rgb"]) and torch.equal(a[0]["T"], c[0]["T"])
    sc1 = scenes.Scene(**{**sc.__dict__})
    pc = sc.mean.astype(np.float64).T @ cam.R_wc.astype(np.float64).T + cam.t_wc.astype(np.float64)
    sc1.kfac = pc[:, 2].copy()
    _, k1, _ = oracle.render(sc1, cams, with_normal_d=False, binning=b)
    assert torch.abs(c[0]["depth"] - k1[0]["kmap"]).max() < 1e-12
    assert torch.abs(c[0]["depth"] - a[0]["depth"]).max() > 1e-4  # the modes differ


# ------------------------------------------------- normal from depth
def _plane_depth(cam, n, d0):
    """Depth map of the world plane n.X = d0 seen by ``cam``."""
    H, W = cam.height, cam.width
    v, u = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    dt = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones_like(u, dtype=float)])
    dw = np.einsum("ij,jhw->ihw", cam.R_cw.astype(np.float64), dt)
    C = cam.C.astype(np.float64)
    return (d0 - n @ C) / np.einsum("i,ihw->hw", n, dw)


def test_normal_from_depth_recovers_plane_normal():
    cam = scenes.orbit_cameras(1, seed=21, resolutions=[(64, 48)])[0]
    n = np.array([0.3, -0.2, 0.9])
    n = cam.R_cw.astype(np.float64) @ n  # tilted, facing the camera
    n /= np.linalg.norm(n)
    C = cam.C.astype(np.float64)
    d0 = n @ C + 2.0 * (1 if n @ cam.R_cw.astype(np.float64)[:, 2] > 0 else -1)
    D = _plane_depth(cam, n, d0)
    assert D.min() > 0
    for steps in ((1, 2), (2, 1), (1, 1), (2, 2)):
        res = orr.depth_to_normal(torch.as_tensor(D), cam, *steps)
        N = res["normal"].numpy()
        ok = res["valid"].numpy()
        assert ok[2:-2, 2:-2].all() and not ok[0].any()
        facing = n if (n @ C - d0) > 0 else -n   # the side the camera is on
        err = np.abs(N[:, ok] - facing[:, None]).max()
        assert err < 1e-9


def test_back_projection_reprojects_to_pixel():
    cam = scenes.orbit_cameras(1, seed=22, resolutions=[(32, 24)])[0]
    rng = np.random.default_rng(0)
    D = rng.uniform(1, 3, size=(24, 32))
    R_cw, C = cam.R_cw.astype(np.float64), cam.C.astype(np.float64)
    R_wc = np.linalg.inv(R_cw)  # exact inverse of the (float32-rounded) rotation
    for (v, u) in [(3, 5), (20, 30), (12, 16)]:
        dt = np.array([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0])
        Pw = R_cw @ (dt * D[v, u]) + C
        pc = R_wc @ (Pw - C)
        assert abs(pc[2] - D[v, u]) < 1e-12
        assert abs(cam.fx * pc[0] / pc[2] + cam.cx - u) < 1e-9
        assert abs(cam.fy * pc[1] / pc[2] + cam.cy - v) < 1e-9


# ------------------------------------------- gradients: autograd vs FD
def _loss(sc, cams, up, binning):
    _, outs, _ = oracle.render(sc, cams, binning=binning)
    tot = 0.0
    for k, r in enumerate(outs):
        tot += float((r["rgb"].numpy() * up["rgb"][k]).sum())
        tot += float((r["depth"].numpy() * up["depth"][k]).sum())
        tot += float((r["normal"].numpy() * up["normal_g"][k]).sum())
        tot += float((r["kmap"].numpy() * up["kmap"][k]).sum())
        tot += float((r["logits"].numpy() * up["logits"][k]).sum())
        tot += float((r["normal_d"].numpy() * up["normal_d"][k]).sum())
    return tot


def test_oracle_gradient_matches_central_differences():
    """The autograd derivative of the oracle equals central finite differences
    of its own forward, away from kinks (FD at h and h/4 must agree)."""
    sc, cams = scenes.small_room(n=400, width=24, height=20, n_sem=2, seed=3,
                                 log_scale_mean=-2.0)
    # make parameters float64-exact so that perturbations are not rounded
    up = scenes.upstream_grads(cams, sc.n_sem, seed=1)
    _, grads, b = oracle.render_and_grad(sc, cams, up)
    rng = np.random.default_rng(0)
    touched = np.unique(b["vals"])
    checked = 0
    for key in ("mean", "quat", "scale", "opacity", "kfac", "sh", "sem"):
        arr = getattr(sc, key)
        tries = 0
        while tries < 6:
            g = int(rng.choice(touched))
            if arr.ndim == 1:
                idx = (g,)
            elif key in ("mean", "quat", "scale"):
                idx = (int(rng.integers(0, arr.shape[0])), g)
            elif key == "sh":
                idx = (g, int(rng.integers(0, arr.shape[1])), int(rng.integers(0, 3)))
            else:
                idx = (g, int(rng.integers(0, arr.shape[1])))
            tries += 1
            x0 = float(arr[idx])

            def fd(h):
                sc64 = scenes.Scene(**{k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v)
                                       for k, v in sc.__dict__.items()})
                a = getattr(sc64, key)
                a[idx] = x0 + h
                lp = _loss(sc64, cams, up, b)
                a[idx] = x0 - h
                lm = _loss(sc64, cams, up, b)
                return (lp - lm) / (2 * h)

            h = 1e-6 * max(1.0, abs(x0))
            f1, f2 = fd(h), fd(h / 4)
            if abs(f1 - f2) > 1e-4 * max(1.0, abs(f1)):
                continue  # a kink inside the stencil: redraw
            an = float(grads[key][idx])
            assert abs(an - f1) <= 1e-5 * max(1.0, abs(f1)), (key, idx, an, f1)
            checked += 1
    assert checked >= 20
