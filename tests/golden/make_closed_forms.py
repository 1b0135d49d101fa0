"""Writes the closed-form fixtures of the oracle pins.

axis_aligned_depth.json: closed-form midpoint depths.  For an axis-aligned
ellipsoid with semi-axes s centred at (0, 0, z0) on the optical axis of a
camera at the origin, the ray (x~, y~, 1) reaches its Mahalanobis-closest point
(the midpoint of the two intersections, Eq. midpoint of Sec. 3.2) at depth
z0 / (1 + s_z^2 (x~^2/s_x^2 + y~^2/s_y^2)).

axis_aligned_render.json: the same closed form at integer pixels of a posed
camera, for rendering one Gaussian end to end.  The camera looks along world
+x (camera-to-world rotation R_cw = 90 degrees about y, a signed permutation,
so every pose entry is exact in float32) from C = (0.5, -0.25, 1.0); the
Gaussian sits at camera-frame (0, 0, z0), i.e. world mu = C + z0 R_cw e_z,
rotated by the same R_cw (quaternion (1, 0, 1, 0), any norm), so its axes are
the camera axes and its semi-axes in the camera frame are s.  Pixel (u, v)
has x~ = (u - cx)/fx, y~ = (v - cy)/fy (Eq. computeRay with the supplement's
back-projection convention), and the expected depth is the formula above.
All inputs are dyadic numbers exact in float32.

Uses only these formulas; nothing here calls the oracle or the library.
"""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def axis_aligned_depth():
    rng = np.random.default_rng(2024)
    cases = []
    for _ in range(24):
        s = np.exp(rng.normal(-2.5, 0.8, 3))
        z0 = float(rng.uniform(1.0, 8.0))
        xt, yt = (float(v) for v in rng.uniform(-0.4, 0.4, 2))
        depth = z0 / (1.0 + s[2] ** 2 * (xt ** 2 / s[0] ** 2 + yt ** 2 / s[1] ** 2))
        cases.append(dict(s=[float(v) for v in s], z0=z0, xt=xt, yt=yt, depth=depth))
    cases.append(dict(s=[0.3, 0.3, 0.3], z0=2.0, xt=0.1, yt=0.2, depth=2.0 / (1 + 0.01 + 0.04)))
    out = dict(source="closed form of the Mahalanobis-closest point on the ray; "
                      "Sec. 3.2 Eq. midpoint and supplement Sec. 1 quadratic",
               cases=cases)
    with open(os.path.join(HERE, "axis_aligned_depth.json"), "w") as f:
        json.dump(out, f, indent=1)


def axis_aligned_render():
    W, H, f = 96, 80, 128.0
    cx, cy = W / 2.0, H / 2.0
    R_cw = [[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]]
    C = [0.5, -0.25, 1.0]
    rng = np.random.default_rng(77)
    cases = []
    for z0, s in ((2.5, (0.09375, 0.0625, 0.125)), (3.25, (0.125, 0.09375, 0.0625)),
                  (4.0, (0.1875, 0.125, 0.25)), (5.5, (0.25, 0.3125, 0.1875))):
        sig_px = min(s[0], s[1]) / z0 * f   # pixel sigma along the short axis
        rad = max(1, int(1.2 * sig_px))
        pix = []
        for _ in range(12):
            du, dv = (int(v) for v in rng.integers(-rad, rad + 1, 2))
            u, v = int(cx) + du, int(cy) + dv
            xt, yt = (u - cx) / f, (v - cy) / f
            depth = z0 / (1.0 + s[2] ** 2 * (xt ** 2 / s[0] ** 2 + yt ** 2 / s[1] ** 2))
            pix.append(dict(u=u, v=v, depth=depth))
        mu = [C[i] + z0 * R_cw[i][2] for i in range(3)]
        cases.append(dict(z0=z0, s=list(s), mu=mu, pixels=pix))
    out = dict(source="closed form of the Mahalanobis-closest point (Sec. 3.2 Eq. midpoint) "
                      "at integer pixels of a posed camera (Eq. computeRay)",
               camera=dict(width=W, height=H, f=f, cx=cx, cy=cy, R_cw=R_cw, C=C),
               quat=[1.0, 0.0, 1.0, 0.0], opacity=0.875, cases=cases)
    with open(os.path.join(HERE, "axis_aligned_render.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    axis_aligned_depth()
    axis_aligned_render()
