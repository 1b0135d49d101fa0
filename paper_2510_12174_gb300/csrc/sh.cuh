// Real spherical-harmonic basis to degree 3 (float32) and its gradient.
//
// The paper stores view-dependent colour as SH coefficients per colour
// channel (Eq. 1) and blends it as 3DGS does; the colour of a Gaussian seen
// from C is max(0, sum_k Y_k(dir) h_k + 1/2), dir = normalize(mu - C).
#pragma once

namespace unigs {

// Real SH constants, each from its closed form (orthonormal real basis,
// no Condon-Shortley phase).
#define SH_C0 0.28209479177387814f    // 1 / (2 sqrt(pi))
#define SH_C1 0.48860251190291992f    // sqrt(3 / (4 pi))
#define SH_C2A 1.0925484305920792f    // sqrt(15 / pi) / 2          (xy, yz, xz)
#define SH_C2B 0.31539156525252005f   // sqrt(5 / pi) / 4           (3z^2 - 1)
#define SH_C2C 0.54627421529603959f   // sqrt(15 / pi) / 4          (x^2 - y^2)
#define SH_C3A 0.59004358992664352f   // sqrt(35 / (2 pi)) / 4      (y(3x^2-y^2), x(x^2-3y^2))
#define SH_C3B 2.8906114426405538f    // sqrt(105 / pi) / 2         (xyz)
#define SH_C3C 0.45704579946446572f   // sqrt(21 / (2 pi)) / 4      (y(5z^2-1), x(5z^2-1))
#define SH_C3D 0.37317633259011546f   // sqrt(7 / pi) / 4           (z(5z^2-3))
#define SH_C3E 1.4453057213202769f    // sqrt(105 / pi) / 4         (z(x^2-y^2))

__device__ __forceinline__ void sh_eval_basis(float x, float y, float z, int deg, float* Y) {
    Y[0] = SH_C0;
    if (deg < 1) return;
    Y[1] = SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = SH_C1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_C2A * x * y;
    Y[5] = SH_C2A * y * z;
    Y[6] = SH_C2B * (3.f * zz - 1.f);
    Y[7] = SH_C2A * x * z;
    Y[8] = SH_C2C * (xx - yy);
    if (deg < 3) return;
    Y[9] = SH_C3A * y * (3.f * xx - yy);
    Y[10] = SH_C3B * x * y * z;
    Y[11] = SH_C3C * y * (5.f * zz - 1.f);
    Y[12] = SH_C3D * z * (5.f * zz - 3.f);
    Y[13] = SH_C3C * x * (5.f * zz - 1.f);
    Y[14] = SH_C3E * z * (xx - yy);
    Y[15] = SH_C3A * x * (xx - 3.f * yy);
}

// Partial derivatives of the basis polynomials w.r.t. (x, y, z).
__device__ __forceinline__ void sh_eval_basis_grad(float x, float y, float z, int deg,
                                                   float (*dY)[3]) {
    for (int k = 0; k < 16; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0.f;
    if (deg < 1) return;
    dY[1][1] = SH_C1;
    dY[2][2] = SH_C1;
    dY[3][0] = SH_C1;
    if (deg < 2) return;
    dY[4][0] = SH_C2A * y; dY[4][1] = SH_C2A * x;
    dY[5][1] = SH_C2A * z; dY[5][2] = SH_C2A * y;
    dY[6][2] = 6.f * SH_C2B * z;
    dY[7][0] = SH_C2A * z; dY[7][2] = SH_C2A * x;
    dY[8][0] = 2.f * SH_C2C * x; dY[8][1] = -2.f * SH_C2C * y;
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[9][0] = 6.f * SH_C3A * x * y; dY[9][1] = SH_C3A * (3.f * xx - 3.f * yy);
    dY[10][0] = SH_C3B * y * z; dY[10][1] = SH_C3B * x * z; dY[10][2] = SH_C3B * x * y;
    dY[11][1] = SH_C3C * (5.f * zz - 1.f); dY[11][2] = 10.f * SH_C3C * y * z;
    dY[12][2] = SH_C3D * (15.f * zz - 3.f);
    dY[13][0] = SH_C3C * (5.f * zz - 1.f); dY[13][2] = 10.f * SH_C3C * x * z;
    dY[14][0] = 2.f * SH_C3E * x * z; dY[14][1] = -2.f * SH_C3E * y * z;
    dY[14][2] = SH_C3E * (xx - yy);
    dY[15][0] = SH_C3A * (3.f * xx - 3.f * yy); dY[15][1] = -6.f * SH_C3A * x * y;
}

}  // namespace unigs
