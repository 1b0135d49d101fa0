"""Algebraic identities the CUDA kernels rely on, checked in float64 on the CPU.

These are not oracle pins: the oracle forms every quantity directly.  They pin
the rewritten forms the kernels evaluate instead, so that a sign or index slip
in a derivation fails here, before any GPU parity test.
"""
import numpy as np
import pytest


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _case(rng):
    """A camera (world->camera R_wc, t_wc), a Gaussian in front of it and a pixel."""
    R_wc = _rot(rng.normal(size=4))
    t_wc = rng.normal(size=3)
    R_cw = R_wc.T
    C = -R_cw @ t_wc
    fx, fy = rng.uniform(300, 1500, size=2)
    cx, cy = rng.uniform(100, 900, size=2)
    p_c = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.5, 40)])
    mu = R_cw @ (p_c - t_wc)
    R = _rot(rng.normal(size=4))
    s = np.exp(rng.normal(-3.5, 1.0, size=3))
    u, v = rng.uniform(0, 1000, size=2)
    return dict(R_wc=R_wc, R_cw=R_cw, C=C, fx=fx, fy=fy, cx=cx, cy=cy, p_c=p_c, mu=mu,
                R=R, s=s, u=u, v=v)


def _setup(k):
    Sinv = np.diag(1.0 / k["s"])
    M = Sinv @ k["R"].T @ k["R_cw"]           # camera ray -> local scaled
    vs = Sinv @ k["R"].T @ (k["C"] - k["mu"])
    d = np.array([(k["u"] - k["cx"]) / k["fx"], (k["v"] - k["cy"]) / k["fy"], 1.0])
    return M, vs, d, M @ d


@pytest.mark.parametrize("seed", range(20))
def test_cross_product_as_two_pixel_offset_vectors(seed):
    """v_s x d_s = dx P1 + dy P2 with (dx, dy) the pixel offset from the
    projected centre and P1_a = kappa_a (M_a2 m_y - M_a1) / fx,
    P2_a = kappa_a (M_a0 - M_a2 m_x) / fy, kappa_a = z s_a / (s_b s_c),
    m = p_c / z the centre's ray (the preprocess's record vectors)."""
    k = _case(np.random.default_rng(seed))
    M, vs, d, ds = _setup(k)
    direct = np.cross(vs, ds)
    z = k["p_c"][2]
    mx, my = k["p_c"][0] / z, k["p_c"][1] / z
    s = k["s"]
    kap = np.array([z * s[0] / (s[1] * s[2]), z * s[1] / (s[0] * s[2]),
                    z * s[2] / (s[0] * s[1])])
    P1 = kap * (M[:, 2] * my - M[:, 1]) / k["fx"]
    P2 = kap * (M[:, 0] - M[:, 2] * mx) / k["fy"]
    dx = k["u"] - (k["fx"] * mx + k["cx"])
    dy = k["v"] - (k["fy"] * my + k["cy"])
    folded = dx * P1 + dy * P2
    scale = np.linalg.norm(vs) * np.linalg.norm(ds)
    assert np.allclose(folded, direct, rtol=0, atol=1e-12 * scale), (folded, direct)


@pytest.mark.parametrize("seed", range(10))
def test_discriminant_by_lagrange(seed):
    """b'^2 - a (|v_s|^2 - 1) = a - |v_s x d_s|^2 (a = |d_s|^2, b' = v_s . d_s):
    the cancellation-free discriminant of the ray-ellipsoid quadratic."""
    k = _case(np.random.default_rng(100 + seed))
    _, vs, _, ds = _setup(k)
    a, bp = ds @ ds, vs @ ds
    cv = np.cross(vs, ds)
    lhs = bp * bp - a * (vs @ vs - 1.0)
    rhs = a - cv @ cv
    assert abs(lhs - rhs) <= 1e-9 * max(bp * bp, a * (vs @ vs))


def _go_index(ns, p, c):
    """Float offset of channel c of pixel row p in the swizzled upstream tile."""
    return p * ns + ((((c >> 2) ^ p) & (ns // 4 - 1)) << 2) + (c & 3)


@pytest.mark.parametrize("ns", [8, 16, 32, 64])
def test_upstream_tile_xor_addresses(ns):
    """The backward reads chunk c of row p at (row base | key) ^ 16 c and the
    gather's step i at (lane base | key) ^ 16 ((i RPS) % LPR) + i RPS NS 4; both
    equal the swizzled offsets for a tile aligned to the row size."""
    lpr, rps = ns // 4, 32 // (ns // 4)
    for base in (ns * 4 * 7, 7168, 1024 + 28 * 256):
        if base % (ns * 4):
            continue
        for p in range(256):
            a_row = (base + p * ns * 4) | ((p & (lpr - 1)) << 4)
            for c in range(lpr):
                assert a_row ^ (c << 4) == base + 4 * _go_index(ns, p, 4 * c)
        for warp in range(8):
            for lane in range(32):
                h, c4 = lane // lpr, lane % lpr
                a_g = (base + (warp * 32 + h) * ns * 4) | ((c4 ^ (h & (lpr - 1))) << 4)
                for i in range(lpr):
                    addr = (a_g ^ (((i * rps) & (lpr - 1)) << 4)) + i * rps * ns * 4
                    want = base + 4 * _go_index(ns, warp * 32 + i * rps + h, 4 * c4)
                    assert addr == want


# --------------------------------------------------------------------------
# Local-frame gradient record of the backward composite.  The pair function
# depends on the Gaussian's rotation R, scale s and centre mu through
# v_s = S^-1 R^T (C - mu) and d_s = S^-1 R^T d.  The kernels accumulate, over
# the pixels of a (camera, Gaussian), the vector g_vs and the matrix
#   B = g_vs (x) w + G2 (x) d_s,   w = v_s + t d_s,   G2 = g_ds - t g_vs,
# which equals g_vs (x) v_s + g_ds (x) d_s for every t; with t the midpoint
# parameter, w is the closest-approach point and G2 is small for a Gaussian
# far from the camera, where g_vs (x) v_s and g_ds (x) d_s are both large and
# cancel.  From B and g_vs:
#   dL/ds_a = -B[a][a] / s_a,  dL/dtheta_k = sum_ij eps_ijk (s_j / s_i) B[i][j]
#   (R -> R exp([theta]_x)),   dL/dmu = -R (g_vs / s).
# --------------------------------------------------------------------------
def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def _ray_loss_torch(vs, ds, up):
    """Depth t = -(v_s.d_s)/(d_s.d_s) and the entry normal of the scaled unit
    sphere (through cv = v_s x d_s, as the kernels differentiate it), dotted
    with fixed upstream weights."""
    import torch
    a = (ds * ds).sum()
    bp = (vs * ds).sum()
    t = -bp / a
    cv = torch.linalg.cross(vs, ds)
    disc = a - (cv * cv).sum()
    pm = torch.linalg.cross(ds, cv) / a
    p = pm - torch.sqrt(disc) / a * ds
    return up[0] * t + (up[1:4] * p).sum()


def test_local_frame_gradient_record_identities():
    import torch
    rng = np.random.default_rng(71)
    eps = np.zeros((3, 3, 3))
    for i, j, k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        eps[i, j, k], eps[j, i, k] = 1.0, -1.0
    n_done = 0
    while n_done < 30:
        R0 = _rot(rng.normal(size=4))
        s = np.exp(rng.normal(-3.5, 1.0, size=3))
        mu = rng.normal(size=3)
        C = mu + rng.normal(size=3) * rng.uniform(0.5, 5.0)
        # a ray through the ellipsoid's silhouette region
        target = mu + R0 @ (s * rng.uniform(-0.8, 0.8, size=3))
        d = target - C
        up = torch.as_tensor(rng.normal(size=4))
        T = lambda x: torch.as_tensor(x, dtype=torch.float64)
        th = torch.zeros(3, dtype=torch.float64, requires_grad=True)
        st = T(s).requires_grad_(True)
        mt = T(mu).requires_grad_(True)
        K = torch.zeros(3, 3, dtype=torch.float64)
        K = K.index_put((torch.tensor([0, 0, 1, 1, 2, 2]), torch.tensor([1, 2, 0, 2, 0, 1])),
                        torch.stack([-th[2], th[1], th[2], -th[0], -th[1], th[0]]))
        R = T(R0) @ torch.linalg.matrix_exp(K)
        vs = (R.T @ (T(C) - mt)) / st
        ds = (R.T @ T(d)) / st
        a = float((ds * ds).sum())
        cv = np.cross(vs.detach().numpy(), ds.detach().numpy())
        if a - cv @ cv <= 1e-3 * a:
            continue
        L = _ray_loss_torch(vs, ds, up)
        g_th, g_s, g_mu = torch.autograd.grad(L, (th, st, mt))
        # the same loss with v_s, d_s as leaves
        vsl = vs.detach().clone().requires_grad_(True)
        dsl = ds.detach().clone().requires_grad_(True)
        g_vs, g_ds = torch.autograd.grad(_ray_loss_torch(vsl, dsl, up), (vsl, dsl))
        g_vs, g_ds = g_vs.numpy(), g_ds.numpy()
        v, dd = vs.detach().numpy(), ds.detach().numpy()
        t = -(v @ dd) / (dd @ dd)
        w = v + t * dd
        B = np.outer(g_vs, w) + np.outer(g_ds - t * g_vs, dd)
        assert np.allclose(B, np.outer(g_vs, v) + np.outer(g_ds, dd), rtol=1e-9,
                           atol=1e-9 * np.abs(np.outer(g_ds, dd)).max())
        assert np.allclose(-np.diag(B) / s, g_s.numpy(), rtol=1e-8, atol=1e-10)
        th_ref = np.einsum("ijk,ij->k", eps, (s[None, :] / s[:, None]) * B)
        assert np.allclose(th_ref, g_th.numpy(), rtol=1e-8, atol=1e-10)
        assert np.allclose(-R0 @ (g_vs / s), g_mu.numpy(), rtol=1e-9, atol=1e-12)
        # the equivalent matrix gradient 1/2 R [g_theta]_x gives the same
        # directional derivative along every tangent R [e]_x
        GR = 0.5 * R0 @ _skew(th_ref)
        for e in np.eye(3):
            assert abs(np.sum(GR * (R0 @ _skew(e))) - th_ref @ e) < 1e-9 * (1 + abs(th_ref @ e))
        # the analytic forms of G2 = g_ds - t g_vs the kernels evaluate: the
        # depth's part is g_bp w (g_bp = -g_t/a), the cross product's g_cv x w
        g_t = float(up[0])
        g_bp = -g_t / a
        depth_vs, depth_ds = g_bp * dd, g_bp * (v + 2 * t * dd)
        assert np.allclose(depth_ds - t * depth_vs, g_bp * w, rtol=1e-9, atol=1e-12)
        g_cv = rng.normal(size=3)
        cv_vs, cv_ds = np.cross(dd, g_cv), np.cross(g_cv, v)
        assert np.allclose(cv_ds - t * cv_vs, np.cross(g_cv, w), rtol=1e-9,
                           atol=1e-9 * np.abs(cv_ds).max())
        n_done += 1


def test_principal_frame_ewa_gradient_identities():
    """The EWA part of the preprocess backward as the kernels evaluate it.

    The gradient record holds G' = E^T G E, the gradient of the 2D covariance
    cov = T Sigma T^T + lowpass I (T = J W, Sigma = R S^2 R^T) in the splat's
    principal frame E (e0 at theta = atan2(2 c01, c00 - c11) / 2).  With
    V' = E^T T R S and H = V'^T G' V', the kernels take
      dL/ds_b = 2 H_bb / s_b,
      dL/dtheta_k = 2 (s_i / s_j - s_j / s_i) H_ij   for (i, j, k) cyclic,
      dL/dT = 2 E (G' V') (R S)^T,
    then J's dependence on the camera-frame centre.  All must equal the
    exact derivative of <G, cov> (rotation R -> R exp([theta]_x))."""
    import torch
    rng = np.random.default_rng(72)
    for _ in range(30):
        R0 = _rot(rng.normal(size=4))
        W = _rot(rng.normal(size=4))
        s = np.exp(rng.normal(-2.5, 1.0, size=3))
        fx, fy = rng.uniform(200, 1500, size=2)
        pc0 = np.array([rng.normal() * 3, rng.normal() * 3, rng.uniform(0.2, 5.0)])
        Gm = rng.normal(size=(2, 2))
        Gm = Gm + Gm.T
        T_ = lambda x: torch.as_tensor(x, dtype=torch.float64)
        th = torch.zeros(3, dtype=torch.float64, requires_grad=True)
        st = T_(s).requires_grad_(True)
        pc = T_(pc0).requires_grad_(True)
        Kx = torch.zeros(3, 3, dtype=torch.float64).index_put(
            (torch.tensor([0, 0, 1, 1, 2, 2]), torch.tensor([1, 2, 0, 2, 0, 1])),
            torch.stack([-th[2], th[1], th[2], -th[0], -th[1], th[0]]))
        R = T_(R0) @ torch.linalg.matrix_exp(Kx)
        Sig = R @ torch.diag(st * st) @ R.T
        x, y, z = pc[0], pc[1], pc[2]
        zero = torch.zeros((), dtype=torch.float64)
        J = torch.stack([torch.stack([fx / z, zero, -fx * x / (z * z)]),
                         torch.stack([zero, fy / z, -fy * y / (z * z)])])
        T = J @ T_(W)
        cov = T @ Sig @ T.T + 0.3 * torch.eye(2, dtype=torch.float64)
        L = (T_(Gm) * cov).sum()
        g_th, g_s, g_pc = torch.autograd.grad(L, (th, st, pc))
        # the kernels' evaluation
        cv = cov.detach().numpy()
        ang = 0.5 * np.arctan2(2 * cv[0, 1], cv[0, 0] - cv[1, 1])
        ec, es = np.cos(ang), np.sin(ang)
        E = np.array([[ec, -es], [es, ec]])
        Gp = E.T @ Gm @ E
        Tn = T.detach().numpy()
        M = R0 * s[None, :]
        Vp = (E.T @ Tn) @ M
        GV = Gp @ Vp
        H = Vp.T @ GV
        gs_k = 2 * np.diag(H) / s
        gth_k = np.array([2 * (s[1] / s[2] - s[2] / s[1]) * H[1, 2],
                          2 * (s[2] / s[0] - s[0] / s[2]) * H[2, 0],
                          2 * (s[0] / s[1] - s[1] / s[0]) * H[0, 1]])
        gT = 2 * (E @ GV) @ M.T
        gJ = gT @ W.T
        iz = 1 / pc0[2]
        gpc_k = np.array([
            gJ[0, 2] * (-fx * iz * iz), gJ[1, 2] * (-fy * iz * iz),
            -gJ[0, 0] * fx * iz * iz + gJ[0, 2] * 2 * fx * pc0[0] * iz ** 3
            - gJ[1, 1] * fy * iz * iz + gJ[1, 2] * 2 * fy * pc0[1] * iz ** 3])
        sc = lambda v: 1e-9 * (1 + np.abs(v).max())
        assert np.allclose(gs_k, g_s.numpy(), rtol=1e-9, atol=sc(g_s.numpy()))
        assert np.allclose(gth_k, g_th.numpy(), rtol=1e-9, atol=sc(g_th.numpy()))
        assert np.allclose(gpc_k, g_pc.numpy(), rtol=1e-9, atol=sc(g_pc.numpy()))
        # E diagonalises the 2D covariance (the frame the record is kept in)
        d = E.T @ cv @ E
        assert abs(d[0, 1]) < 1e-9 * np.abs(cv).max()


def test_conditional_form_of_the_quadratic():
    """The double-float alpha path of ill-conditioned splats evaluates
    q = D^T K D (K = cov^-1) in the conditional (LDL^T) form the preprocess
    records: pivot on y when c00 >= c11,
      q = P (dy + rho dx)^2 + e dx^2,  P = c00 / det, rho = -c01 / c00,
      e = 1 / c00,
    on x otherwise (the roles of x and y swapped), and u = K D from the same
    quantities: u_pivot = P w, u_other = P w rho + e b.  Exact in float64 for
    every conditioning, including the near-singular covariances that send a
    splat down that path."""
    rng = np.random.default_rng(73)
    for _ in range(2000):
        th = rng.uniform(0, np.pi)
        l1, l2 = np.exp(rng.uniform(-2, 12, size=2))
        E = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        cov = E @ np.diag([l1, l2]) @ E.T + 0.3 * np.eye(2)
        c00, c01, c11 = cov[0, 0], cov[0, 1], cov[1, 1]
        det = c00 * c11 - c01 * c01
        K = np.linalg.inv(cov)
        D = rng.normal(size=2) * np.sqrt(max(l1, l2)) * 3
        piv_x = c11 > c00
        cp = c11 if piv_x else c00
        P, rho, e = cp / det, -c01 / cp, 1.0 / cp
        a, b = (D[0], D[1]) if piv_x else (D[1], D[0])
        w = a + rho * b
        q = P * w * w + e * b * b
        q_ref = D @ K @ D
        assert abs(q - q_ref) <= 1e-9 * abs(q_ref) + 1e-12
        assert abs(rho) <= 1.0 + 1e-15 and P > 0 and e > 0
        ua, ub = P * w, P * w * rho + e * b
        u = np.array([ua, ub]) if piv_x else np.array([ub, ua])
        assert np.allclose(u, K @ D, rtol=1e-9, atol=1e-12 * np.abs(K @ D).max())
