// Double-float EWA projection of one Gaussian (Sec. 3.1 follows 3DGS's EWA
// splatting): camera-frame centre, Jacobian terms and the projected scaled
// axes V = J R_wc R S, the 2x3 factor of the 2D covariance V V^T, from which
// the preprocess derives the centre, the conic (and its conditional form),
// the principal axes and, for the preprocess backward, the short-axis row of
// V in that frame.
#pragma once

#include "ff.cuh"
#include "unigs_internal.cuh"

namespace unigs {

struct EwaFF {
    ff pc[3];      // camera-frame centre
    ff xz, yz;     // x / z, y / z
    ff V[2][3];    // J R_wc R S
};

__device__ __forceinline__ void ewa_ff(const DevCam& cam, float mux, float muy, float muz,
                                       float qw, float qx, float qy, float qz, float sx,
                                       float sy, float sz, EwaFF& o) {
    const float* W = cam.R_wc;
    ff* pc = o.pc;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        pc[i] = ff_add(ff_add(ff_add(two_prod(W[3 * i], mux), two_prod(W[3 * i + 1], muy)),
                              two_prod(W[3 * i + 2], muz)),
                       ff_from(cam.t_wc[i]));
    const ff n2 = ff_add(ff_add(two_prod(qw, qw), two_prod(qx, qx)),
                         ff_add(two_prod(qy, qy), two_prod(qz, qz)));
    const ff qn = ff_sqrt(n2);
    const ff w = ff_div(ff_from(qw), qn), x = ff_div(ff_from(qx), qn),
             y = ff_div(ff_from(qy), qn), z = ff_div(ff_from(qz), qn);
    const ff one = ff_from(1.f);
    ff R[3][3];
    R[0][0] = ff_sub(one, ff_scale(ff_add(ff_mul(y, y), ff_mul(z, z)), 2.f));
    R[0][1] = ff_scale(ff_sub(ff_mul(x, y), ff_mul(w, z)), 2.f);
    R[0][2] = ff_scale(ff_add(ff_mul(x, z), ff_mul(w, y)), 2.f);
    R[1][0] = ff_scale(ff_add(ff_mul(x, y), ff_mul(w, z)), 2.f);
    R[1][1] = ff_sub(one, ff_scale(ff_add(ff_mul(x, x), ff_mul(z, z)), 2.f));
    R[1][2] = ff_scale(ff_sub(ff_mul(y, z), ff_mul(w, x)), 2.f);
    R[2][0] = ff_scale(ff_sub(ff_mul(x, z), ff_mul(w, y)), 2.f);
    R[2][1] = ff_scale(ff_add(ff_mul(y, z), ff_mul(w, x)), 2.f);
    R[2][2] = ff_sub(one, ff_scale(ff_add(ff_mul(x, x), ff_mul(y, y)), 2.f));
    const float s[3] = {sx, sy, sz};
    ff M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = ff_mul_f(R[i][j], s[j]);
    const ff iz = ff_div(one, pc[2]);
    const ff xz = ff_mul(pc[0], iz), yz = ff_mul(pc[1], iz);
    o.xz = xz;
    o.yz = yz;
    const ff J00 = ff_mul_f(iz, cam.fx), J11 = ff_mul_f(iz, cam.fy);
    const ff J02 = ff_neg(ff_mul(J00, xz)), J12 = ff_neg(ff_mul(J11, yz));
    // V = T M with T = J R_wc (2x3); cov = V V^T + lowpass I
    ff T[2][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T[0][j] = ff_add(ff_mul_f(J00, W[j]), ff_mul_f(J02, W[6 + j]));
        T[1][j] = ff_add(ff_mul_f(J11, W[3 + j]), ff_mul_f(J12, W[6 + j]));
    }
    ff(&V)[2][3] = o.V;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            V[i][j] = ff_add(ff_add(ff_mul(T[i][0], M[0][j]), ff_mul(T[i][1], M[1][j])),
                             ff_mul(T[i][2], M[2][j]));
}

}  // namespace unigs
