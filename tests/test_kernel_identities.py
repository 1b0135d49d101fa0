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
