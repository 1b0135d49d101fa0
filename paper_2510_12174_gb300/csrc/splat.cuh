// Per-(pixel, Gaussian) math shared by the forward and backward composites.
#pragma once

#include "ff.cuh"
#include "unigs_internal.cuh"

namespace unigs {

// alpha = min(alpha_max, opacity * exp(-1/2 D^T conic D)), D = pixel - centre,
// with the centre held as integer part + remainder.  A pixel outside the
// Gaussian's 3-sigma square (|D_x| > r or |D_y| > r, r of the binning recipe)
// gets -1, below every alpha_min: the Gaussian is not drawn there (the tiles
// of the binning only have to cover the square, so the image does not depend
// on the tile shape).  Ill-conditioned splats (flag set by the preprocess)
// take D exactly as a double-float pair and the quadratic form in its
// conditional form q = P w^2 + e b^2, w = a + rho b (a the pivot coordinate,
// see the record): both terms are non-negative, so only w needs an
// error-free product and sum, where A dx^2 + 2 B dx dy + C dy^2 cancels along
// the long axis; *w_out returns w for splat_kdelta (0 on the float path).
// The branch is uniform across a CTA because all its threads walk the same
// Gaussian.  Written with non-contractible intrinsics so the forward and the
// backward (which recomputes alpha to undo T) obtain the same bits.
__device__ __forceinline__ float splat_alpha(const float* __restrict__ rc, float uf, float vf,
                                             float alpha_max, float* dx_out, float* dy_out,
                                             float* gauss_out, float* w_out) {
    const float ux = __fsub_rn(uf, rc[R_MXH]);  // exact (integers)
    const float vy = __fsub_rn(vf, rc[R_MYH]);
    const float r3 = rc[R_R3];
    float q, w = 0.f;
    bool outside;
    if (rc[R_FLAG] != 0.f) {
        // |ux| >= 1 > |remainder| or ux = 0: the fast transformation is exact
        const ff dx = fast_two_sum(ux, -rc[R_MXL]);
        const ff dy = fast_two_sum(vy, -rc[R_MYL]);
        *dx_out = dx.hi;
        *dy_out = dy.hi;
        outside = fmaxf(fabsf(dx.hi), fabsf(dy.hi)) > r3;
        const bool piv_x = rc[R_CLO + 1] != 0.f;
        const ff a = piv_x ? dx : dy, b = piv_x ? dy : dx;
        const float rh = rc[R_CON + 1], rl = rc[R_CON + 2];
        const ff p = two_prod(rh, b.hi);
        const ff sm = two_sum(a.hi, p.hi);
        const float tail = __fadd_rn(__fadd_rn(sm.lo, p.lo),
                                     __fmaf_rn(rh, b.lo, __fmaf_rn(rl, b.hi, a.lo)));
        w = __fadd_rn(sm.hi, tail);
        q = __fmaf_rn(__fmul_rn(rc[R_CON], w), w, __fmul_rn(__fmul_rn(rc[R_CLO], b.hi), b.hi));
    } else {
        const float dx = __fsub_rn(ux, rc[R_MXL]);
        const float dy = __fsub_rn(vy, rc[R_MYL]);
        *dx_out = dx;
        *dy_out = dy;
        outside = fmaxf(fabsf(dx), fabsf(dy)) > r3;
        const float A = rc[R_CON], B = rc[R_CON + 1], C = rc[R_CON + 2];
        q = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(A, dx), dx), __fmul_rn(__fmul_rn(C, dy), dy)),
                      __fmul_rn(2.f, __fmul_rn(__fmul_rn(B, dx), dy)));
    }
    *w_out = w;
    // the square test is applied as a select, after the exponential, so the
    // warp does not diverge ahead of it
    const float G = __expf(__fmul_rn(-0.5f, q));
    *gauss_out = outside ? 0.f : G;
    return outside ? -1.f : fminf(alpha_max, __fmul_rn(rc[R_OP], G));
}

// u = K D (conic times pixel offset), the direction of every alpha gradient:
// dL/dm = g u and dL/dcov = g/2 u u^T for g = dL/dpower.  For an
// ill-conditioned splat from the conditional form (the gradient of q/2):
// u_a = P w, u_b = P w rho + e b, with w from splat_alpha.
__device__ __forceinline__ void splat_kdelta(const float* __restrict__ rc, float dx, float dy,
                                             float w, float* ux, float* uy) {
    if (rc[R_FLAG] != 0.f) {
        const bool piv_x = rc[R_CLO + 1] != 0.f;
        const float ua = rc[R_CON] * w;
        const float ub = fmaf(ua, rc[R_CON + 1], rc[R_CLO] * (piv_x ? dy : dx));
        *ux = piv_x ? ua : ub;
        *uy = piv_x ? ub : ua;
    } else {
        *ux = fmaf(rc[R_CON], dx, rc[R_CON + 1] * dy);
        *uy = fmaf(rc[R_CON + 1], dx, rc[R_CON + 2] * dy);
    }
}

// a*b - c*d with Kahan's FMA compensation (error about one ulp of the result).
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}

// Ray-ellipsoid quantities of one pair (Sec. 3.2 and the supplement's Sec. 1),
// in the local scaled frame, for the camera-frame ray d~ = (xt, yt, 1):
//   d_s = M_c d~, a = d_s.d_s, b' = v_s.d_s (b = 2b'), t_mid = -b'/a (the
//   depth, because d~_z = 1), cv = v_s x d_s, disc = b'^2 - a c = a - |cv|^2
//   (Lagrange's identity; free of the b^2 - 4ac cancellation),
//   p_mid = (d_s x cv)/a (closest approach), h = sqrt(disc)/a (0 on a miss),
//   p = p_mid - sr h d_s (entry point; exit point when the camera is inside,
//   sr = -1), normal n = sign * normalize(N_w p).
// cv is not formed as v_s x d_s: for a Gaussian far from the camera |v_s| is
// hundreds and the product cancels to the ray's offset from the centre, so
// the float32 rounding of v_s (a few ulp of |v_s|) would move the silhouette
// and the normal.  With v_s = -S^-1 Q p_c, d_s = S^-1 Q d~ (Q = R^T R_cw,
// M_c = S^-1 Q) and p_c = z m~ (m~ = the centre's ray, m~_z = 1):
//   v_s x d_s = det(S^-1) S Q (d~ x p_c) = kappa (.) M_c (Delta x m~),
// Delta = d~ - m~ = ((u - m_x)/fx, (v - m_y)/fy, 0), kappa_a = z s_a / (s_b s_c).
// Delta x m~ is linear in the exactly formed pixel offset (dx, dy) of the
// splat, so the preprocess folds everything else into two vectors of the
// record: cv = dx P1 + dy P2, no cancellation.
// Square root by the approximate hardware instruction (a few ulp; subnormal
// inputs supported): the pair geometry feeds tolerance-checked outputs only.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct PairGeom {
    float ds[3], a, bp, t, cv[3], disc, pm[3], h, p[3], m[3], inv_m, sr;
    bool hit, inside;
};

// dxp, dyp: the pixel offset from the projected centre (splat_alpha's
// outputs).
__device__ __forceinline__ void pair_geometry(const float* __restrict__ rc, float xt, float yt,
                                              float dxp, float dyp, PairGeom& G) {
    const float* M = rc + R_MC;
    const float* vs = rc + R_VS;
#pragma unroll
    for (int i = 0; i < 3; ++i) G.ds[i] = fmaf(M[3 * i], xt, fmaf(M[3 * i + 1], yt, M[3 * i + 2]));
    G.a = fmaf(G.ds[0], G.ds[0], fmaf(G.ds[1], G.ds[1], G.ds[2] * G.ds[2]));
    G.bp = fmaf(vs[0], G.ds[0], fmaf(vs[1], G.ds[1], vs[2] * G.ds[2]));
    const float inv_a = __fdividef(1.f, G.a);  // a = |d_s|^2 > 0, far below 2^126
    G.t = -G.bp * inv_a;
#pragma unroll
    for (int i = 0; i < 3; ++i) G.cv[i] = fmaf(dxp, rc[R_P1 + i], dyp * rc[R_P2 + i]);
    const float cc = fmaf(G.cv[0], G.cv[0], fmaf(G.cv[1], G.cv[1], G.cv[2] * G.cv[2]));
    G.disc = G.a - cc;
    // d_s and cv are orthogonal, so the cross product does not cancel
    G.pm[0] = fmaf(G.ds[1], G.cv[2], -G.ds[2] * G.cv[1]) * inv_a;
    G.pm[1] = fmaf(G.ds[2], G.cv[0], -G.ds[0] * G.cv[2]) * inv_a;
    G.pm[2] = fmaf(G.ds[0], G.cv[1], -G.ds[1] * G.cv[0]) * inv_a;
    // camera inside the 1-sigma ellipsoid (|v_s| <= 1): a per-Gaussian sign
    G.sr = rc[R_SR];
    G.inside = G.sr < 0.f;
    G.hit = G.disc > 0.f;
    G.h = G.hit ? sqrt_approx(G.disc) * inv_a : 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) G.p[i] = fmaf(-G.sr * G.h, G.ds[i], G.pm[i]);
    const float* N = rc + R_NW;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        G.m[i] = fmaf(N[3 * i], G.p[0], fmaf(N[3 * i + 1], G.p[1], N[3 * i + 2] * G.p[2]));
    G.inv_m = rsqrtf(fmaf(G.m[0], G.m[0], fmaf(G.m[1], G.m[1], G.m[2] * G.m[2])));
}

}  // namespace unigs
