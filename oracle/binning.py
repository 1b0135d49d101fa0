"""Tile binning of the oracle: which (tile, Gaussian) pairs exist, and their order.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package.

The paper extends the tile-based pipeline of 3DGS (Sec. 3.4, "Tile-based
Forward Rasterization") and gives no detail of it; the discrete part of that
pipeline (projected centre, 2D covariance with the 0.3 px low-pass, the 3-sigma
radius, the tile rectangle and the depth key) is therefore fixed here as an
explicit IEEE float32 recipe.  Every operation below is a single
correctly-rounded float32 operation (numpy never contracts a*b+c into an FMA),
in the order written, so that any implementation that performs the same
operations in the same order obtains the same bits.  No transcendental
function appears in the recipe.

The recipe, per (camera, Gaussian); (+) and (*) are float32 add and multiply:

  p_c   = R_wc mu + t_wc            row i: ((R_i0*mx + R_i1*my) + R_i2*mz) + t_i
  cull  if not p_c.z > z_near
  qn2   = ((w*w + x*x) + y*y) + z*z ;  cull if not qn2 > 0
  qn    = sqrt(qn2) ; (w,x,y,z) /= qn          (correctly rounded sqrt, divide)
  R(q)  = [[1-2(y*y+z*z), 2(x*y-w*z),   2(x*z+w*y)],
           [2(x*y+w*z),   1-2(x*x+z*z), 2(y*z-w*x)],
           [2(x*z-w*y),   2(y*z+w*x),   1-2(x*x+y*y)]]
  M     = R diag(s)                 M_ij = R_ij * s_j
  Sigma = M M^T                     S_ij = (M_i0*M_j0 + M_i1*M_j1) + M_i2*M_j2
  iz    = 1 / p_c.z
  J00 = fx*iz, J11 = fy*iz, J02 = -(J00*(px*iz)), J12 = -(J11*(py*iz))
  T     = J R_wc                    T_0j = J00*W_0j + J02*W_2j ; T_1j = J11*W_1j + J12*W_2j
  U     = T Sigma                   U_ij = (T_i0*S_0j + T_i1*S_1j) + T_i2*S_2j
  c00 = (U00*T00 + U01*T01) + U02*T02, c01 = (U00*T10 + U01*T11) + U02*T12,
  c11 = (U10*T10 + U11*T11) + U12*T12
  a = c00 + 0.3 ; b = c01 ; c = c11 + 0.3           (EWA low-pass filter)
  det = a*c - b*b ; cull if not det > 0
  mid = 0.5*(a + c) ; lam = mid + sqrt(max(0.1, mid*mid - det))
  r   = ceil(3 * sqrt(lam))                          (3-sigma radius, pixels)
  m_x = fx*(px*iz) + cx ; m_y = fy*(py*iz) + cy     (projected centre)
  rect: x0 = clamp(floor((m_x - r) / TW), 0, TX), x1 = clamp(ceil((m_x + r) / TW), 0, TX)
        (same for y with TH and TY); cull if the rectangle is empty
  key  = (global tile id << 32) | float32 bits of p_c.z

Opacity-aware tile test.  Alg. 2 skips a Gaussian at a pixel where its alpha
is below 1/255, so a (tile, Gaussian) pair only has to be listed when alpha
can reach 1/255 somewhere in the tile.  With the float32 conic
kA = c/det, kB = -(b/det), kC = a/det and q(D) = D^T K D, alpha >= 1/255
needs q <= 2 ln(255 opacity).  The recipe bounds the logarithm from above
without a transcendental: 255*op = m 2^e with m in [1, 2) (exact), and
ln(255 op) <= e*LN2 + (m - 1) (ln m <= m - 1), so
  qlim = (2 (e*LN2 + (m - 1))) * 1.01 + 0.05      (LN2 = float32(ln 2), margin
                                                  for float32 evaluation)
and a rectangle tile is kept iff the minimum of q over the tile's pixel-centre
rectangle [TW tx, TW tx + TW-1] x [TH ty, TH ty + TH-1] is <= qlim.  That minimum is 0 when
the centre lies in the square, else the least of the four edge minima: on a
vertical edge x = xe, dx = xe - m_x, dy = clamp(-(kB*dx)/kC, Y0 - m_y, Y1 - m_y)
(and symmetrically on horizontal edges), q = ((kA*dx)*dx + ((2*kB)*dx)*dy)
+ (kC*dy)*dy.  Strongly elongated splats, (a + c)^2 > 4096 det, keep every
tile of their rectangle (float32 cannot resolve their minimum reliably).  The
culled pairs have alpha < 1/255 at every pixel of the tile, so the rendered
result is the one the full rectangle gives.

Within a tile the list is ordered by (depth bits, Gaussian index): a stable
sort by the 64-bit key of the instances emitted in (camera, Gaussian, tile
row-major) order.

Tiles are TW x TH pixels (16 x 16 by default; the library also takes 8 x 32,
32 x 8 and 64 x 4), TX = ceil(W / TW) and TY = ceil(H / TH) per camera.  The
divisions by TW and TH are by powers of two, hence exact.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32
TILE = 16
DEFAULT_TILE = (TILE, TILE)


def _rect_axis(m, r, n_tiles, side):
    lo = np.floor((m - r) / f32(side))
    hi = np.ceil((m + r) / f32(side))
    nt = f32(n_tiles)
    lo = np.fmin(np.fmax(lo, f32(0)), nt)
    hi = np.fmin(np.fmax(hi, f32(0)), nt)
    return lo.astype(np.int64), hi.astype(np.int64)


LN2_F32 = f32(0.6931471805599453)


def tile_keep(pr, g, tx, ty):
    """Opacity-aware tile test for Gaussian indices ``g`` and tile coordinates
    (arrays of equal length), float32 recipe of the module docstring."""
    mx, my = pr["mean2d"][0][g], pr["mean2d"][1][g]
    kA, kB, kC = pr["conic32"][0][g], pr["conic32"][1][g], pr["conic32"][2][g]
    qlim = pr["qlim"][g]
    tw, th = pr["tile"]
    X0 = (tx * tw).astype(f32)
    X1 = (tx * tw + (tw - 1)).astype(f32)
    Y0 = (ty * th).astype(f32)
    Y1 = (ty * th + (th - 1)).astype(f32)
    two = f32(2)
    with np.errstate(all="ignore"):
        def qf(dx, dy):
            return ((kA * dx) * dx + ((two * kB) * dx) * dy) + (kC * dy) * dy

        def vert(xe):
            dx = xe - mx
            dy = np.fmin(np.fmax(-(kB * dx) / kC, Y0 - my), Y1 - my)
            return qf(dx, dy)

        def horiz(ye):
            dy = ye - my
            dx = np.fmin(np.fmax(-(kB * dy) / kA, X0 - mx), X1 - mx)
            return qf(dx, dy)

        qmin = np.fmin(np.fmin(vert(X0), vert(X1)), np.fmin(horiz(Y0), horiz(Y1)))
        inside = (X0 <= mx) & (mx <= X1) & (Y0 <= my) & (my <= Y1)
        qmin = np.where(inside, f32(0), qmin)
    return pr["no_cull"][g] | (qmin <= qlim)


def project_fp32(scene, cam, tile=DEFAULT_TILE) -> dict:
    """Float32 recipe for one camera with tiles of tile = (TW, TH) pixels.
    Returns per-Gaussian arrays."""
    tile_w, tile_h = int(tile[0]), int(tile[1])
    with np.errstate(all="ignore"):
        mu = scene.mean.astype(f32)
        Rw = cam.R_wc.astype(f32)
        tw = cam.t_wc.astype(f32)
        p = [((Rw[i, 0] * mu[0] + Rw[i, 1] * mu[1]) + Rw[i, 2] * mu[2]) + tw[i]
             for i in range(3)]
        px, py, pz = p
        in_front = pz > f32(cam.z_near)

        w, x, y, z = [scene.quat[i].astype(f32) for i in range(4)]
        qn2 = ((w * w + x * x) + y * y) + z * z
        qok = qn2 > f32(0)
        qn = np.sqrt(qn2)
        w, x, y, z = w / qn, x / qn, y / qn, z / qn
        one, two = f32(1), f32(2)
        R = [[one - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y)],
             [two * (x * y + w * z), one - two * (x * x + z * z), two * (y * z - w * x)],
             [two * (x * z - w * y), two * (y * z + w * x), one - two * (x * x + y * y)]]
        s = [scene.scale[j].astype(f32) for j in range(3)]
        M = [[R[i][j] * s[j] for j in range(3)] for i in range(3)]
        S = [[None] * 3 for _ in range(3)]
        for i in range(3):
            for j in range(i, 3):
                S[i][j] = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2]
                S[j][i] = S[i][j]
        iz = one / pz
        fx, fy = f32(cam.fx), f32(cam.fy)
        cx, cy = f32(cam.cx), f32(cam.cy)
        J00 = fx * iz
        J11 = fy * iz
        xz = px * iz
        yz = py * iz
        J02 = -(J00 * xz)
        J12 = -(J11 * yz)
        T = [[J00 * Rw[0, j] + J02 * Rw[2, j] for j in range(3)],
             [J11 * Rw[1, j] + J12 * Rw[2, j] for j in range(3)]]
        U = [[(T[i][0] * S[0][j] + T[i][1] * S[1][j]) + T[i][2] * S[2][j]
              for j in range(3)] for i in range(2)]
        c00 = (U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2]
        c01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2]
        c11 = (U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2]
        a = c00 + f32(0.3)
        b = c01
        c = c11 + f32(0.3)
        det = a * c - b * b
        det_ok = det > f32(0)
        mid = f32(0.5) * (a + c)
        lam = mid + np.sqrt(np.fmax(f32(0.1), mid * mid - det))
        r = np.ceil(f32(3) * np.sqrt(lam))
        mx = fx * xz + cx
        my = fy * yz + cy
        TX = (cam.width + tile_w - 1) // tile_w
        TY = (cam.height + tile_h - 1) // tile_h
        x0, x1 = _rect_axis(mx, r, TX, tile_w)
        y0, y1 = _rect_axis(my, r, TY, tile_h)
        valid = in_front & qok & det_ok & (x1 > x0) & (y1 > y0)
        # opacity-aware tile test (module docstring)
        kA = c / det
        kB = -(b / det)
        kC = a / det
        ac = a + c
        no_cull = (ac * ac) > (f32(4096) * det)
        y = f32(255) * scene.opacity.astype(f32)
        mant, ex = np.frexp(y)             # y = mant * 2^ex, mant in [0.5, 1)
        m = (mant * two).astype(f32)       # exact
        e = (ex - 1).astype(f32)
        lnb = e * LN2_F32 + (m - one)
        qlim = (two * lnb) * f32(1.01) + f32(0.05)
    zbits = pz.astype(f32).view(np.uint32)
    pr = dict(p_c=np.stack(p), z=pz, zbits=zbits, cov2d=np.stack([a, b, c]),
              det=det, radius=r, mean2d=np.stack([mx, my]),
              rect=np.stack([x0, x1, y0, y1]), valid=valid, tiles_x=TX, tiles_y=TY,
              conic32=np.stack([kA, kB, kC]), qlim=qlim, no_cull=no_cull, tile=(tile_w, tile_h))
    # tiles kept per Gaussian
    touched = np.zeros(pz.shape[0], dtype=np.int64)
    idx = np.nonzero(valid)[0]
    if idx.size:
        gg, tx, ty = _rect_tiles(pr, idx)
        keep = tile_keep(pr, gg, tx, ty)
        touched = np.bincount(gg[keep], minlength=pz.shape[0]).astype(np.int64)
    pr["touched"] = touched
    return pr


def _rect_tiles(pr, idx):
    """All (Gaussian, tx, ty) of the rectangles of Gaussians ``idx``, in
    (Gaussian, row-major tile) order."""
    x0, x1, y0, y1 = [v.astype(np.int64) for v in pr["rect"][:, idx]]
    wdt = x1 - x0
    cnt = wdt * (y1 - y0)
    rep = np.repeat(np.arange(idx.size), cnt)
    first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    local = np.arange(rep.size) - first[rep]
    ty = y0[rep] + local // wdt[rep]
    tx = x0[rep] + local % wdt[rep]
    return idx[rep], tx, ty


def bin_cameras(scene, cams, tile=DEFAULT_TILE) -> dict:
    """Binning over several cameras with global tile ids.

    Camera k's tiles are numbered tile_offset[k] + ty * TX_k + tx.  Returns the
    sorted 64-bit keys, the Gaussian index of each instance (``vals``), the
    per-tile [start, end) ranges, the per-camera projections and the tile
    shape.
    """
    projs = [project_fp32(scene, c, tile) for c in cams]
    tile_off = [0]
    for pr in projs:
        tile_off.append(tile_off[-1] + pr["tiles_x"] * pr["tiles_y"])
    keys_l, vals_l = [], []
    for k, pr in enumerate(projs):
        idx = np.nonzero(pr["valid"])[0]
        x0, x1, y0, y1 = pr["rect"][:, idx]
        TX = pr["tiles_x"]
        for g, a0, a1, b0, b1 in zip(idx, x0, x1, y0, y1):
            ty, tx = np.meshgrid(np.arange(b0, b1), np.arange(a0, a1), indexing="ij")
            ty, tx = ty.ravel(), tx.ravel()
            keep = tile_keep(pr, np.full(ty.size, g), tx, ty)
            ty, tx = ty[keep], tx[keep]
            tiles = (tile_off[k] + ty * TX + tx).ravel().astype(np.uint64)
            keys_l.append((tiles << np.uint64(32)) | np.uint64(pr["zbits"][g]))
            vals_l.append(np.full(tiles.size, g, dtype=np.uint32))
    if keys_l:
        keys = np.concatenate(keys_l)
        vals = np.concatenate(vals_l)
    else:
        keys = np.zeros(0, np.uint64)
        vals = np.zeros(0, np.uint32)
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    n_tiles = tile_off[-1]
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    starts = np.searchsorted(tiles, np.arange(n_tiles), side="left")
    ends = np.searchsorted(tiles, np.arange(n_tiles), side="right")
    ranges = np.stack([starts, ends], axis=1).astype(np.uint32)
    return dict(keys=keys, vals=vals, ranges=ranges, tile_offset=np.array(tile_off),
                projs=projs, tile=tuple(int(t) for t in tile))


def bin_cameras_fast(scene, cams, tile=DEFAULT_TILE) -> dict:
    """Same result as :func:`bin_cameras`, vectorised for large scenes."""
    projs = [project_fp32(scene, c, tile) for c in cams]
    tile_off = [0]
    for pr in projs:
        tile_off.append(tile_off[-1] + pr["tiles_x"] * pr["tiles_y"])
    keys_l, vals_l = [], []
    for k, pr in enumerate(projs):
        idx = np.nonzero(pr["valid"])[0]
        if idx.size == 0:
            continue
        gg, tx, ty = _rect_tiles(pr, idx)
        keep = tile_keep(pr, gg, tx, ty)
        gg, tx, ty = gg[keep], tx[keep], ty[keep]
        tiles = (tile_off[k] + ty * pr["tiles_x"] + tx).astype(np.uint64)
        keys_l.append((tiles << np.uint64(32)) | pr["zbits"][gg].astype(np.uint64))
        vals_l.append(gg.astype(np.uint32))
    keys = np.concatenate(keys_l) if keys_l else np.zeros(0, np.uint64)
    vals = np.concatenate(vals_l) if vals_l else np.zeros(0, np.uint32)
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    n_tiles = tile_off[-1]
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    starts = np.searchsorted(tiles, np.arange(n_tiles), side="left")
    ends = np.searchsorted(tiles, np.arange(n_tiles), side="right")
    ranges = np.stack([starts, ends], axis=1).astype(np.uint32)
    return dict(keys=keys, vals=vals, ranges=ranges, tile_offset=np.array(tile_off),
                projs=projs, tile=tuple(int(t) for t in tile))
