"""Real spherical-harmonic basis up to degree 3, float64 (oracle).

TEST INFRASTRUCTURE ONLY.

The paper stores view-dependent colour as SH coefficients h per colour channel
(Eq. 1, the map representation) and blends the colour "consistent with 3DGS"
(Sec. 7 of the supplement).  The colour of a Gaussian seen from camera centre
C is max(0, sum_k Y_k(dir) h_k + 1/2) with dir = normalize(mu - C).

The basis is the orthonormal real SH basis, written as polynomials of the unit
direction (x, y, z), without the Condon-Shortley phase, in the band order
m = -l..l.  Each normalising constant is derived here from its closed form
(K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) folded into the polynomial),
not taken from a table; tests check orthonormality by quadrature.
"""
from __future__ import annotations

import math

import torch

PI = math.pi
C0 = 0.5 / math.sqrt(PI)                     # 1/(2 sqrt(pi))
C1 = math.sqrt(3.0 / (4.0 * PI))
C2_xy = 0.5 * math.sqrt(15.0 / PI)           # xy, yz, xz
C2_z = 0.25 * math.sqrt(5.0 / PI)            # 3z^2 - 1
C2_x2y2 = 0.25 * math.sqrt(15.0 / PI)        # x^2 - y^2
C3_a = 0.25 * math.sqrt(35.0 / (2.0 * PI))   # y(3x^2-y^2), x(x^2-3y^2)
C3_b = 0.5 * math.sqrt(105.0 / PI)           # xyz
C3_c = 0.25 * math.sqrt(21.0 / (2.0 * PI))   # y(5z^2-1), x(5z^2-1)
C3_d = 0.25 * math.sqrt(7.0 / PI)            # z(5z^2-3)
C3_e = 0.25 * math.sqrt(105.0 / PI)          # z(x^2-y^2)


def sh_basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """Basis values for unit directions ``dirs`` [..., 3] -> [..., (degree+1)^2]."""
    x, y, z = dirs[..., 0], dirs[..., 1], dirs[..., 2]
    out = [torch.full_like(x, C0)]
    if degree >= 1:
        out += [C1 * y, C1 * z, C1 * x]
    if degree >= 2:
        out += [C2_xy * x * y, C2_xy * y * z, C2_z * (3.0 * z * z - 1.0),
                C2_xy * x * z, C2_x2y2 * (x * x - y * y)]
    if degree >= 3:
        out += [C3_a * y * (3.0 * x * x - y * y), C3_b * x * y * z,
                C3_c * y * (5.0 * z * z - 1.0), C3_d * z * (5.0 * z * z - 3.0),
                C3_c * x * (5.0 * z * z - 1.0), C3_e * z * (x * x - y * y),
                C3_a * x * (x * x - 3.0 * y * y)]
    return torch.stack(out, dim=-1)
