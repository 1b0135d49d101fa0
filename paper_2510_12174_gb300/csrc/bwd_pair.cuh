// Per-(pixel, Gaussian) body of the backward composite (Alg. 4), shared by
// the FP32-pipe kernel and the tensor-core kernel: everything but the semantic
// dot product, which each kernel forms its own way.
#pragma once

#include "splat.cuh"

namespace unigs {

// Upstream gradients of one pixel (every channel but the logits).
struct PixelUp {
    float rgb[3], D, N[3], K;
};

// Loads a pixel's upstream gradients (absent channels stay zero).
__device__ __forceinline__ void load_pixel_up(const unigs_grad_outputs& go, int64_t pix,
                                              int64_t HW, int64_t idx, PixelUp& up) {
    if (go.rgb)
#pragma unroll
        for (int c = 0; c < 3; ++c) up.rgb[c] = go.rgb[pix * 3 + c * HW + idx];
    if (go.depth) up.D = go.depth[pix + idx];
    if (go.normal_g)
#pragma unroll
        for (int c = 0; c < 3; ++c) up.N[c] = go.normal_g[pix * 3 + c * HW + idx];
    if (go.kmap) up.K = go.kmap[pix + idx];
}

__device__ __forceinline__ void cross_acc(const float* a, const float* b, float* c) {
    c[0] += a[1] * b[2] - a[2] * b[1];
    c[1] += a[2] * b[0] - a[0] * b[2];
    c[2] += a[0] * b[1] - a[1] * b[0];
}

// One pair of the reverse walk.  With w_i = alpha_i T_i,
// G_i = upstream gradient . features of Gaussian i (G_sem its logit part) and
// S_i = sum_{j>i} w_j G_j (Sacc),
//   dL/dx_i,ch = w_i g_ch, dL/dalpha_i = T_i G_i - S_i / (1 - alpha_i).
// Restores T across the Gaussian (T <- T / (1 - alpha)) where the pixel
// contributes, advances Sacc and fills the pair's 32-entry gradient vector gv
// (every entry zero where it does not: w = 0 and dL/dalpha = 0, all
// intermediates finite).  alpha, (dx, dy), Gs and wq come from splat_alpha.
// Returns w (0 where the pixel does not contribute).
__device__ __forceinline__ float bwd_pair(const float* __restrict__ rc, const PixelUp& up,
                                          float xt, float yt, float wq, float dx,
                                          float dy, float alpha, float Gs, bool contrib,
                                          float G_sem, float alpha_max, int center_depth,
                                          float& T, float& Sacc, float (&gv)[32]) {
    const float om = 1.f - alpha;
    // om >= 1 - alpha_max.  The restoration T <- T / om runs along
    // the whole list, so it keeps the correctly rounded division
    // (with an approximate quotient the worst cancelling rotation
    // gradient of a 200k-Gaussian test scene drifted 2.5x further
    // from the float64 reference); dL/dalpha takes an approximate
    // reciprocal
    const float rom = __fdividef(1.f, om);
    if (contrib) T = __fdiv_rn(T, om);
    const float w = contrib ? alpha * T : 0.f;
    PairGeom G;
    pair_geometry(rc, xt, yt, dx, dy, G);
    const float depth = center_depth ? rc[R_Z] : G.t;
    const float sg = G.inside ? -1.f : 1.f;
    float nh[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) nh[i] = G.m[i] * G.inv_m;
    // G_i: upstream gradient . features of Gaussian i
    const float Gi = up.rgb[0] * rc[R_RGB] + up.rgb[1] * rc[R_RGB + 1] +
                     up.rgb[2] * rc[R_RGB + 2] + up.D * depth + up.K * rc[R_K] +
                     sg * (up.N[0] * nh[0] + up.N[1] * nh[1] + up.N[2] * nh[2]) +
                     G_sem;
    const float dL_da = contrib ? T * Gi - Sacc * rom : 0.f;
    Sacc = fmaf(w, Gi, Sacc);
    // alpha = min(alpha_max, op * Gs)
    const bool clamped = rc[R_OP] * Gs > alpha_max;
    const float g_pow = clamped ? 0.f : dL_da * alpha;
    gv[G_OP] = clamped ? 0.f : dL_da * Gs;
    // power = -1/2 D^T K D: dL/dm = g u, dL/dcov = g/2 u u^T, u = K D
    float kux, kuy;
    splat_kdelta(rc, dx, dy, wq, &kux, &kuy);
    {
        // dL/dcov = 1/2 g u u^T, recorded in the splat's principal frame E
        // (u' = E^T u): in the pixel frame the entries of a thin splat seen far
        // off-axis are dominated by the short axis and would cancel in the
        // preprocess backward, which maps them back onto the projected 3D axes
        const float pu = fmaf(rc[R_EC], kux, rc[R_ES] * kuy);
        const float pv = fmaf(-rc[R_ES], kux, rc[R_EC] * kuy);
        gv[G_CA] = 0.5f * g_pow * pu * pu;
        gv[G_CB] = g_pow * pu * pv;
        gv[G_CC] = 0.5f * g_pow * pv * pv;
    }
    gv[G_MX] = kux * g_pow;
    gv[G_MY] = kuy * g_pow;
    gv[G_RGB] = w * up.rgb[0];
    gv[G_RGB + 1] = w * up.rgb[1];
    gv[G_RGB + 2] = w * up.rgb[2];
    gv[G_K] = w * up.K;
    const float* Nw = rc + R_NW;
    const float inv_a = __fdividef(1.f, G.a);
    // The Gaussian enters through v_s and d_s.  Besides g_vs the
    // record takes B = g_vs (x) w + G2 (x) d_s with w = v_s + t d_s
    // (the closest-approach point p_mid, formed without
    // cancellation) and G2 = g_ds - t g_vs, which is small and is
    // formed here term by term: g_vs (x) v_s and g_ds (x) d_s are
    // both large for a Gaussian far from the camera and would cancel
    // in the scale and rotation gradients (B equals their sum).
    // g_a collects the normal's dependence on a = d_s.d_s only.
    float g_vs[3] = {0.f, 0.f, 0.f}, g2[3] = {0.f, 0.f, 0.f}, g_a = 0.f;
    // depth t_mid = -b'/a: g_vs = g_bp d_s, g_ds = g_bp (v_s + 2 t d_s),
    // so its part of G2 is g_bp w
    const float g_t = w * up.D;
    gv[G_Z] = center_depth ? g_t : 0.f;
    if (!center_depth) {
        const float g_bp = -g_t * inv_a;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            g_vs[i] = g_bp * G.ds[i];
            g2[i] = g_bp * G.pm[i];
        }
    }
    // normal n = sg * m / |m|, m = N_w p
    const float gn[3] = {w * up.N[0], w * up.N[1], w * up.N[2]};
    const float dgn = gn[0] * nh[0] + gn[1] * nh[1] + gn[2] * nh[2];
    float g_m[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) g_m[i] = sg * (gn[i] - dgn * nh[i]) * G.inv_m;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) gv[G_NW + 3 * r + c] = g_m[r] * G.p[c];
    float g_p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        g_p[c] = Nw[c] * g_m[0] + Nw[3 + c] * g_m[1] + Nw[6 + c] * g_m[2];
    // p = p_mid - sr h d_s, h = sqrt(disc)/a
    float g_disc = 0.f;
    if (G.hit) {
        const float g_h = -G.sr * (g_p[0] * G.ds[0] + g_p[1] * G.ds[1] +
                                   g_p[2] * G.ds[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) g2[i] -= G.sr * G.h * g_p[i];
        // dh/ddisc = 1 / (2 a sqrt(disc))
        g_disc = 0.5f * g_h * inv_a * rsqrtf(G.disc);
        g_a -= g_h * G.h * inv_a;
    }
    // disc = a - |cv|^2
    g_a += g_disc;
    float g_cv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) g_cv[i] = -2.f * g_disc * G.cv[i];
    // p_mid = (d_s x cv) / a
    const float g_q[3] = {g_p[0] * inv_a, g_p[1] * inv_a, g_p[2] * inv_a};
    cross_acc(G.cv, g_q, g2);
    cross_acc(g_q, G.ds, g_cv);
    g_a -= (g_p[0] * G.pm[0] + g_p[1] * G.pm[1] + g_p[2] * G.pm[2]) * inv_a;
    // cv = v_s x d_s: g_vs += d_s x g_cv, and g_ds += g_cv x v_s,
    // whose part of G2 is g_cv x v_s - t (d_s x g_cv) = g_cv x w
    cross_acc(G.ds, g_cv, g_vs);
    cross_acc(g_cv, G.pm, g2);
    // a = d_s . d_s
#pragma unroll
    for (int i = 0; i < 3; ++i) g2[i] = fmaf(2.f * g_a, G.ds[i], g2[i]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            gv[G_B + 3 * r + c] = fmaf(g_vs[r], G.pm[c], g2[r] * G.ds[c]);
        gv[G_VS + r] = g_vs[r];
    }
    return w;
}

}  // namespace unigs
