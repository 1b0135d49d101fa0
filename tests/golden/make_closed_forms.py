"""Writes axis_aligned_depth.json: closed-form midpoint depths.

For an axis-aligned ellipsoid with semi-axes s centred at (0, 0, z0) on the
optical axis of a camera at the origin, the ray (x~, y~, 1) reaches its
Mahalanobis-closest point (the midpoint of the two intersections, Eq. midpoint
of Sec. 3.2) at depth z0 / (1 + s_z^2 (x~^2/s_x^2 + y~^2/s_y^2)).  Uses only this
formula; nothing here calls the oracle or the library.
"""
import json
import os

import numpy as np

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
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "axis_aligned_depth.json"), "w") as f:
    json.dump(out, f, indent=1)
