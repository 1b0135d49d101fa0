// Preprocess, in two kernels.  The culling pass takes one thread per (camera,
// Gaussian): the binning recipe, the opacity-aware tile count and the list of
// pairs with a kept tile.  The splat pass takes one thread per listed pair:
// the continuous setup below and the record.  Culled pairs would otherwise
// leave most lanes of a warp idle through the long double-float chain.
//
// Discrete part (projected centre, EWA 2D covariance with the 0.3 px
// low-pass, 3-sigma radius, tile rectangle, depth key) follows a fixed
// float32 recipe: each operation is a single correctly rounded float32
// operation in a fixed order (the __f*_rn intrinsics are never contracted
// into FMAs), so the tile lists are bit-reproducible.  The paper extends the
// tile pipeline of 3DGS without detailing it (Sec. 3.4).
//
// Continuous part: conic, a compensated projected centre (integer part plus
// a float remainder, so alpha is evaluated from an accurate pixel offset),
// SH colour (real SH basis to degree 3, colour = max(0, Y.h + 1/2)), and the
// ray-ellipsoid setup of Sec. 3.2: v_s = S^-1 R^T (C - mu) and the map from
// the camera-frame pixel ray d~ = ((u-cx)/fx, (v-cy)/fy, 1) to the local
// scaled direction, d_s = S^-1 R^T R_cw d~ = M_c d~; plus N_w = R S^-1, which
// maps a scaled-local surface point to the world-frame ellipsoid normal.
#include "ewa_ff.cuh"
#include "launch.h"
#include "ff.cuh"
#include "sh.cuh"

namespace unigs {

// Shorthands for the exactly-rounded, never-contracted float32 operations of
// the binning recipe.
#define RM(a, b) __fmul_rn((a), (b))
#define RA(a, b) __fadd_rn((a), (b))
#define RS(a, b) __fsub_rn((a), (b))

struct Recipe {
    float px, py, pz;       // camera-frame centre
    float R[3][3];          // rotation of the normalised quaternion
    float a, b, c, det;     // 2D covariance (+ low-pass) and determinant
    float mx, my, radius;   // projected centre and 3-sigma radius
    int x0, x1, y0, y1;     // tile rectangle [x0,x1) x [y0,y1)
    bool valid;
};

__device__ __forceinline__ void rect_axis(float m, float r, int n_tiles, int side, int* lo,
                                          int* hi) {
    // side is a power of two, so multiplying by its exact reciprocal gives
    // the bits of the division
    const float nt = (float)n_tiles, inv = 1.f / (float)side;
    float l = floorf(__fmul_rn(RS(m, r), inv));
    float h = ceilf(__fmul_rn(RA(m, r), inv));
    l = fminf(fmaxf(l, 0.f), nt);
    h = fminf(fmaxf(h, 0.f), nt);
    *lo = (int)l;
    *hi = (int)h;
}

__device__ __forceinline__ void binning_recipe(const DevCam& cam, float mx_, float my_, float mz_,
                                               float qw, float qx, float qy, float qz, float sx,
                                               float sy, float sz, float lowpass, Recipe& o) {
    const float* W = cam.R_wc;
    o.px = RA(RA(RA(RM(W[0], mx_), RM(W[1], my_)), RM(W[2], mz_)), cam.t_wc[0]);
    o.py = RA(RA(RA(RM(W[3], mx_), RM(W[4], my_)), RM(W[5], mz_)), cam.t_wc[1]);
    o.pz = RA(RA(RA(RM(W[6], mx_), RM(W[7], my_)), RM(W[8], mz_)), cam.t_wc[2]);
    const bool in_front = o.pz > cam.z_near;

    const float qn2 = RA(RA(RA(RM(qw, qw), RM(qx, qx)), RM(qy, qy)), RM(qz, qz));
    const bool qok = qn2 > 0.f;
    const float qn = __fsqrt_rn(qn2);
    const float w = __fdiv_rn(qw, qn), x = __fdiv_rn(qx, qn), y = __fdiv_rn(qy, qn),
                z = __fdiv_rn(qz, qn);
    float (&R)[3][3] = o.R;
    R[0][0] = RS(1.f, RM(2.f, RA(RM(y, y), RM(z, z))));
    R[0][1] = RM(2.f, RS(RM(x, y), RM(w, z)));
    R[0][2] = RM(2.f, RA(RM(x, z), RM(w, y)));
    R[1][0] = RM(2.f, RA(RM(x, y), RM(w, z)));
    R[1][1] = RS(1.f, RM(2.f, RA(RM(x, x), RM(z, z))));
    R[1][2] = RM(2.f, RS(RM(y, z), RM(w, x)));
    R[2][0] = RM(2.f, RS(RM(x, z), RM(w, y)));
    R[2][1] = RM(2.f, RA(RM(y, z), RM(w, x)));
    R[2][2] = RS(1.f, RM(2.f, RA(RM(x, x), RM(y, y))));

    const float s[3] = {sx, sy, sz};
    float M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = RM(R[i][j], s[j]);
    float S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            S[i][j] = RA(RA(RM(M[i][0], M[j][0]), RM(M[i][1], M[j][1])), RM(M[i][2], M[j][2]));
            S[j][i] = S[i][j];
        }
    const float iz = __fdiv_rn(1.f, o.pz);
    const float J00 = RM(cam.fx, iz);
    const float J11 = RM(cam.fy, iz);
    const float xz = RM(o.px, iz);
    const float yz = RM(o.py, iz);
    const float J02 = -RM(J00, xz);
    const float J12 = -RM(J11, yz);
    float T[2][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T[0][j] = RA(RM(J00, W[0 * 3 + j]), RM(J02, W[2 * 3 + j]));
        T[1][j] = RA(RM(J11, W[1 * 3 + j]), RM(J12, W[2 * 3 + j]));
    }
    float U[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            U[i][j] = RA(RA(RM(T[i][0], S[0][j]), RM(T[i][1], S[1][j])), RM(T[i][2], S[2][j]));
    const float c00 = RA(RA(RM(U[0][0], T[0][0]), RM(U[0][1], T[0][1])), RM(U[0][2], T[0][2]));
    const float c01 = RA(RA(RM(U[0][0], T[1][0]), RM(U[0][1], T[1][1])), RM(U[0][2], T[1][2]));
    const float c11 = RA(RA(RM(U[1][0], T[1][0]), RM(U[1][1], T[1][1])), RM(U[1][2], T[1][2]));
    o.a = RA(c00, lowpass);
    o.b = c01;
    o.c = RA(c11, lowpass);
    o.det = RS(RM(o.a, o.c), RM(o.b, o.b));
    const bool det_ok = o.det > 0.f;
    const float mid = RM(0.5f, RA(o.a, o.c));
    const float lam = RA(mid, __fsqrt_rn(fmaxf(0.1f, RS(RM(mid, mid), o.det))));
    o.radius = ceilf(RM(3.f, __fsqrt_rn(lam)));
    o.mx = RA(RM(cam.fx, xz), cam.cx);
    o.my = RA(RM(cam.fy, yz), cam.cy);
    rect_axis(o.mx, o.radius, cam.tiles_x, cam.tile_w, &o.x0, &o.x1);
    rect_axis(o.my, o.radius, cam.tiles_y, cam.tile_h, &o.y0, &o.y1);
    o.valid = in_front && qok && det_ok && (o.x1 > o.x0) && (o.y1 > o.y0);
}

#undef RM
#undef RA
#undef RS

// Double-float splat setup from the float32 inputs: camera-frame centre,
// projected centre f (x/z) + c split as integer part + remainder, and the
// conic (inverse of J W Sigma W^T J^T + lowpass I).  The float32 recipe above
// only decides the tile rectangle; the continuous quantities that alpha needs
// are computed here to about 48 bits, because an elongated splat far from its
// centre makes the quadratic form cancel by orders of magnitude.
struct SplatFF {
    float mxh, myh, mxl, myl;
    ff A, B, C;
    float kappa;
    float cxx, cyy;  // diagonal of the 2D covariance
    float ec, es;    // principal axis e0 = (ec, es) of the 2D covariance
    float lam0, lam1;  // its eigenvalues along e0 (the larger) and e1
    float vp1[3];      // e1^T V: the short-axis row of the projected scaled axes
    // conditional form of the quadratic, q = P (a + rho b)^2 + e b^2 with the
    // pivot coordinate a = x when c11 > c00 (piv_x), else a = y
    float P, e;
    ff rho;
    bool piv_x;
};

__device__ __forceinline__ void split_center(ff m, float* hi, float* lo) {
    const float h = rintf(m.hi);
    *hi = h;
    *lo = __fadd_rn(__fsub_rn(m.hi, h), m.lo);  // m.hi - h is exact
}

__device__ __forceinline__ void splat_ff(const DevCam& cam, float mux, float muy, float muz,
                                         float qw, float qx, float qy, float qz, float sx,
                                         float sy, float sz, float lowpass, SplatFF& o) {
    EwaFF e;
    ewa_ff(cam, mux, muy, muz, qw, qx, qy, qz, sx, sy, sz, e);
    const ff(&V)[2][3] = e.V;
    const ff xz = e.xz, yz = e.yz;
    const ff lp = ff_from(lowpass);
    const ff c00 = ff_add(ff_add(ff_add(ff_mul(V[0][0], V[0][0]), ff_mul(V[0][1], V[0][1])),
                                 ff_mul(V[0][2], V[0][2])), lp);
    const ff c11 = ff_add(ff_add(ff_add(ff_mul(V[1][0], V[1][0]), ff_mul(V[1][1], V[1][1])),
                                 ff_mul(V[1][2], V[1][2])), lp);
    const ff c01 = ff_add(ff_add(ff_mul(V[0][0], V[1][0]), ff_mul(V[0][1], V[1][1])),
                          ff_mul(V[0][2], V[1][2]));
    const ff det = ff_sub(ff_mul(c00, c11), ff_mul(c01, c01));
    o.cxx = ff_val(c00);
    o.cyy = ff_val(c11);
    // principal axes: e0 at theta = atan2(2 c01, c00 - c11) / 2 (any
    // orthonormal pair is a valid frame; this one keeps the recorded
    // covariance gradient free of cancellation for thin splats)
    sincosf(0.5f * atan2f(2.f * ff_val(c01), ff_val(ff_sub(c00, c11))), &o.es, &o.ec);
    // e1^T V in double-float, rounded: the preprocess backward's projected
    // scaled axes along the short axis, orders of magnitude below V's entries
    // for a thin splat seen far off-axis
#pragma unroll
    for (int j = 0; j < 3; ++j)
        o.vp1[j] = ff_val(ff_add(ff_mul_f(V[0][j], -o.es), ff_mul_f(V[1][j], o.ec)));
    {
        const float hd = 0.5f * ff_val(ff_sub(c00, c11)), co = ff_val(c01);
        o.lam0 = 0.5f * (ff_val(c00) + ff_val(c11)) + sqrtf(hd * hd + co * co);
        o.lam1 = ff_val(det) / o.lam0;
    }
    o.A = ff_div(c11, det);
    o.B = ff_neg(ff_div(c01, det));
    o.C = ff_div(c00, det);
    // pivot on the coordinate with the larger conic diagonal: for a = y,
    // P = c00 / det, rho = -c01 / c00 (|rho| <= 1), e = 1 / c00 (only P
    // carries the determinant's cancellation, held in double-float)
    o.piv_x = ff_val(c11) > ff_val(c00);
    const ff cp = o.piv_x ? c11 : c00;
    o.P = ff_val(ff_div(cp, det));
    o.rho = ff_neg(ff_div(c01, cp));
    o.e = __frcp_rn(ff_val(cp));
    split_center(ff_add(ff_mul_f(xz, cam.fx), ff_from(cam.cx)), &o.mxh, &o.mxl);
    split_center(ff_add(ff_mul_f(yz, cam.fy), ff_from(cam.cy)), &o.myh, &o.myl);
    // eigenvalue ratio of the conic: lmax^2 / det(conic)
    const float a = o.A.hi, b = o.B.hi, c = o.C.hi;
    const float lmax = 0.5f * (a + c) + sqrtf(0.25f * (a - c) * (a - c) + b * b);
    const float detK = 1.f / ff_val(det);
    o.kappa = lmax * lmax / fmaxf(detK, 1e-30f);
}

// Opacity-aware tile-test inputs from the float32 recipe: conic, and
// qlim = 2 (e LN2 + (m - 1)) * 1.01 + 0.05 with 255 op = m 2^e, m in [1, 2)
// (an upper bound of 2 ln(255 op), the q at which alpha falls to 1/255).
__device__ __forceinline__ void cull_record(const Recipe& rc, float op, float* cr) {
    cr[C_MX] = rc.mx;
    cr[C_MY] = rc.my;
    cr[C_KA] = __fdiv_rn(rc.c, rc.det);
    cr[C_KB] = -__fdiv_rn(rc.b, rc.det);
    cr[C_KC] = __fdiv_rn(rc.a, rc.det);
    const float ac = __fadd_rn(rc.a, rc.c);
    cr[C_NOCULL] = (__fmul_rn(ac, ac) > __fmul_rn(4096.f, rc.det)) ? 1.f : 0.f;
    int ex = 0;
    const float mant = frexpf(__fmul_rn(255.f, op), &ex);
    const float m = __fmul_rn(mant, 2.f);
    const float e = (float)(ex - 1);
    const float lnb = __fadd_rn(__fmul_rn(e, 0x1.62e43p-1f), __fsub_rn(m, 1.f));
    cr[C_QLIM] = __fadd_rn(__fmul_rn(__fmul_rn(2.f, lnb), 1.01f), 0.05f);
    cr[7] = 0.f;
}

// Number of kept tiles of the rectangle [x0,x1) x [y0,y1) (opacity-aware test)
// for tiles of tw x th pixels.
__device__ __forceinline__ uint32_t count_kept_serial(const float* cr, int x0, int x1, int y0,
                                                      int y1, int tw, int th) {
    uint32_t kept = 0;
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) kept += tile_keep(cr, tx, ty, tw, th) ? 1u : 0u;
    return kept;
}


__global__ void __launch_bounds__(256)
    preprocess_kernel(const unigs_gaussians g, const CamTable* __restrict__ tab, int n_cams,
                      int tw, int th, float lowpass, uint2* __restrict__ rect,
                      uint32_t* __restrict__ touched, uint32_t* __restrict__ zbits,
                      float* __restrict__ cull, WsHeader* __restrict__ hdr,
                      uint32_t* __restrict__ kept_list) {
    const int64_t n = g.n;
    const int64_t total = n * (int64_t)n_cams;
    const int lane = threadIdx.x & 31;
    // the loop bound is uniform across the block, so whole warps iterate
    // together and can test large rectangles cooperatively
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const bool act = t < total;
        const int k = act ? (int)(t / n) : 0;
        const int64_t i = act ? t - (int64_t)k * n : 0;
        const DevCam& cam = tab->cam[k];
        Recipe rc = {};
        float cr[CULL_FLOATS] = {};
        float mux = 0.f, muy = 0.f, muz = 0.f, qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f;
        float sx = 1.f, sy = 1.f, sz = 1.f;
        int nt = 0;
        if (act) {
            mux = __ldg(g.mean + i); muy = __ldg(g.mean + n + i); muz = __ldg(g.mean + 2 * n + i);
            qw = __ldg(g.quat + i); qx = __ldg(g.quat + n + i);
            qy = __ldg(g.quat + 2 * n + i); qz = __ldg(g.quat + 3 * n + i);
            sx = __ldg(g.scale + i); sy = __ldg(g.scale + n + i); sz = __ldg(g.scale + 2 * n + i);
            binning_recipe(cam, mux, muy, muz, qw, qx, qy, qz, sx, sy, sz, lowpass, rc);
            if (rc.valid) {
                cull_record(rc, __ldg(g.opacity + i), cr);
                nt = (rc.x1 - rc.x0) * (rc.y1 - rc.y0);
            }
        }
        uint32_t kept = (nt > 0 && nt <= COOP_TILES)
                            ? count_kept_serial(cr, rc.x0, rc.x1, rc.y0, rc.y1, tw, th) : 0u;
        unsigned big = __ballot_sync(0xffffffffu, nt > COOP_TILES);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            float cb[CULL_FLOATS];
#pragma unroll
            for (int q = 0; q < CULL_FLOATS; ++q) cb[q] = __shfl_sync(0xffffffffu, cr[q], src);
            const int bx0 = __shfl_sync(0xffffffffu, rc.x0, src);
            const int by0 = __shfl_sync(0xffffffffu, rc.y0, src);
            const int bw = __shfl_sync(0xffffffffu, rc.x1 - rc.x0, src);
            const int bn = __shfl_sync(0xffffffffu, nt, src);
            uint32_t cnt = 0;
            for (int j0 = 0; j0 < bn; j0 += 32) {
                const int j = j0 + lane;
                const bool keep = j < bn && tile_keep(cb, bx0 + j % bw, by0 + j / bw, tw, th);
                cnt += __popc(__ballot_sync(0xffffffffu, keep));
            }
            if (lane == src) kept = cnt;
        }
        // the pairs with a kept tile go to the splat setup, appended warp by
        // warp (one atomic per warp) so that its warps run full
        const bool push = act && rc.valid && kept != 0;
        const unsigned pm = __ballot_sync(0xffffffffu, push);
        if (pm) {
            uint32_t slot = 0;
            if (lane == 0) slot = atomicAdd(&hdr->n_kept, (uint32_t)__popc(pm));
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (push) kept_list[slot + __popc(pm & ((1u << lane) - 1u))] = (uint32_t)t;
        }
        if (!act) continue;
        if (!rc.valid) {
            touched[t] = 0;
            rect[t] = make_uint2(0, 0);
            zbits[t] = __float_as_uint(rc.pz);
            continue;
        }
        touched[t] = kept;
        rect[t] = make_uint2((uint32_t)rc.x0 | ((uint32_t)rc.x1 << 16),
                             (uint32_t)rc.y0 | ((uint32_t)rc.y1 << 16));
        zbits[t] = __float_as_uint(rc.pz);
        float4* cdst = reinterpret_cast<float4*>(cull + (size_t)t * CULL_FLOATS);
        cdst[0] = make_float4(cr[0], cr[1], cr[2], cr[3]);
        cdst[1] = make_float4(cr[4], cr[5], cr[6], cr[7]);
    }
}

// Splat setup of the pairs with a kept tile (the list the culling pass
// appended): the double-float conic and centre, the principal axes, the SH
// colour and the ray-ellipsoid record.  The binning recipe is recomputed (the
// same bits as in the culling pass) for the rotation, depth and radius.
__global__ void __launch_bounds__(256)
    preprocess_splat_kernel(const unigs_gaussians g, const CamTable* __restrict__ tab,
                            float lowpass, const uint32_t* __restrict__ kept_list,
                            const WsHeader* __restrict__ hdr, const float* __restrict__ cull,
                            float* __restrict__ rec, float4* __restrict__ vp) {
    const int64_t n = g.n;
    const int64_t n_kept = hdr->n_kept;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_kept;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = kept_list[idx];
        const int k = (int)(t / n);
        const int64_t i = t - (int64_t)k * n;
        const DevCam& cam = tab->cam[k];
        const float mux = __ldg(g.mean + i), muy = __ldg(g.mean + n + i),
                    muz = __ldg(g.mean + 2 * n + i);
        const float qw = __ldg(g.quat + i), qx = __ldg(g.quat + n + i),
                    qy = __ldg(g.quat + 2 * n + i), qz = __ldg(g.quat + 3 * n + i);
        const float sx = __ldg(g.scale + i), sy = __ldg(g.scale + n + i),
                    sz = __ldg(g.scale + 2 * n + i);
        Recipe rc;
        binning_recipe(cam, mux, muy, muz, qw, qx, qy, qz, sx, sy, sz, lowpass, rc);
        const float qlim = cull[(size_t)t * CULL_FLOATS + C_QLIM];

        float o[REC_FLOATS];
        SplatFF sf;
        splat_ff(cam, mux, muy, muz, qw, qx, qy, qz, sx, sy, sz, lowpass, sf);
        o[R_MXH] = sf.mxh;
        o[R_MYH] = sf.myh;
        o[R_MXL] = sf.mxl;
        o[R_MYL] = sf.myl;
        o[R_OP] = __ldg(g.opacity + i);
        o[R_K] = __ldg(g.kfac + i);
        o[R_FLAG] = sf.kappa > KAPPA_FF ? 1.f : 0.f;
        if (o[R_FLAG] != 0.f) {
            // ill-conditioned: the conditional form (see splat_alpha)
            o[R_CON + 0] = sf.P;
            o[R_CON + 1] = sf.rho.hi;
            o[R_CON + 2] = sf.rho.lo;
            o[R_CLO + 0] = sf.e;
            o[R_CLO + 1] = sf.piv_x ? 1.f : 0.f;
        } else {
            o[R_CON + 0] = sf.A.hi;
            o[R_CON + 1] = sf.B.hi;
            o[R_CON + 2] = sf.C.hi;
            o[R_CLO + 0] = 0.f;
            o[R_CLO + 1] = 0.f;
        }
        o[R_CLO + 2] = 0.f;
        o[R_EC] = sf.ec;
        o[R_ES] = sf.es;

        // colour from SH, viewing direction mu - C
        float dx = mux - cam.C[0], dy = muy - cam.C[1], dz = muz - cam.C[2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16];
        const int deg = g.sh_degree;
        const int n_sh = (deg + 1) * (deg + 1);
        sh_eval_basis(dx, dy, dz, deg, Y);
        float col[3] = {0.5f, 0.5f, 0.5f};
        const size_t shb = (size_t)i * n_sh * 3;
        for (int kk = 0; kk < n_sh; ++kk)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                col[ch] = fmaf(Y[kk], load_feat(g.sh, shb + kk * 3 + ch, g.feat_dtype), col[ch]);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) o[R_RGB + ch] = fmaxf(col[ch], 0.f);

        // ray-ellipsoid setup (Sec. 3.2)
        const float is[3] = {1.f / sx, 1.f / sy, 1.f / sz};
        const float e[3] = {cam.C[0] - mux, cam.C[1] - muy, cam.C[2] - muz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // row a of S^-1 R^T: column a of R scaled by 1/s_a
            const float ra0 = rc.R[0][a], ra1 = rc.R[1][a], ra2 = rc.R[2][a];
#pragma unroll
            for (int b = 0; b < 3; ++b)
                o[R_MC + a * 3 + b] =
                    is[a] * fmaf(ra0, cam.R_cw[0 * 3 + b],
                                 fmaf(ra1, cam.R_cw[1 * 3 + b], ra2 * cam.R_cw[2 * 3 + b]));
            o[R_VS + a] = is[a] * fmaf(ra0, e[0], fmaf(ra1, e[1], ra2 * e[2]));
#pragma unroll
            for (int b = 0; b < 3; ++b) o[R_NW + a * 3 + b] = rc.R[a][b] * is[b];
        }
        o[R_Z] = rc.pz;
        {
            // v_s x d_s without cancellation (see pair_geometry): with
            // Q = R^T R_cw, M_c = S^-1 Q and p_c = z m~ (m~ = p_c / z, the
            // centre's ray), v_s x d_s = det(S^-1) S Q (d~ x p_c)
            // = kappa (.) M_c (Delta x m~), kappa_a = z s_a / (s_b s_c), where
            // Delta = d~ - m~ = (dx / fx, dy / fy, 0) for the pixel offset
            // (dx, dy) from the projected centre.  Delta x m~ = (Dy, -Dx,
            // Dx m~_y - Dy m~_x) is linear in (dx, dy), so the product is
            // dx P1 + dy P2 with
            //   P1_a = kappa_a (M_a2 m~_y - M_a1) / fx,
            //   P2_a = kappa_a (M_a0 - M_a2 m~_x) / fy.
            const float iz = 1.f / rc.pz;
            const float mtx = rc.px * iz, mty = rc.py * iz;
            const float kap[3] = {rc.pz * sx / (sy * sz), rc.pz * sy / (sx * sz),
                                  rc.pz * sz / (sx * sy)};
            const float ifx = 1.f / cam.fx, ify = 1.f / cam.fy;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float* Ma = o + R_MC + 3 * a;
                o[R_P1 + a] = kap[a] * fmaf(Ma[2], mty, -Ma[1]) * ifx;
                o[R_P2 + a] = kap[a] * fmaf(-Ma[2], mtx, Ma[0]) * ify;
            }
            o[R_R3] = rc.radius;
        }
        {
            const float* v = o + R_VS;
            const float vv = fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2]));
            o[R_SR] = vv <= 1.f ? -1.f : 1.f;
        }
        {
            // box of the q <= qlim ellipse (x half-extent sqrt(qlim * Sigma_xx)),
            // with a relative and a one-pixel margin, clipped to the 3-sigma
            // square (plus a margin far above the float32 error of the centre)
            const float ql = fmaxf(qlim, 0.f);
            const float sq = rc.radius + 0.01f;
            o[R_EXTX] = fminf(sqrtf(ql * sf.cxx) * 1.01f + 1.f, sq);
            o[R_EXTY] = fminf(sqrtf(ql * sf.cyy) * 1.01f + 1.f, sq);
            // the same ellipse's half-extents along its principal axes
            o[R_E0] = sqrtf(ql * sf.lam0) * 1.01f + 1.f;
            o[R_E1] = sqrtf(ql * fmaxf(sf.lam1, 0.f)) * 1.01f + 1.f;
        }
        vp[t] = make_float4(sf.vp1[0], sf.vp1[1], sf.vp1[2], 0.f);
        float4* dst = reinterpret_cast<float4*>(rec + (size_t)t * REC_FLOATS);
#pragma unroll
        for (int q = 0; q < REC_FLOATS / 4; ++q)
            dst[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
}

__global__ void init_kernel(CamTable tab, int n_cams, CamTable* __restrict__ dst,
                            WsHeader* __restrict__ hdr) {
    const int k = threadIdx.x;
    if (k < n_cams) dst->cam[k] = tab.cam[k];
    if (k == 0) {
        hdr->status = 0;
        hdr->n_instances = 0;
        hdr->need = 0;
        hdr->n_eval = 0;
        hdr->n_blend = 0;
        hdr->nonfinite = 0;
        hdr->n_kept = 0;
    }
}

__global__ void sem_tail_kernel(const __nv_bfloat16* __restrict__ src, float* __restrict__ dst) {
    *dst = __bfloat162float(*src);
}

// bfloat16 semantic rows -> float32 copy in the workspace (exact), so the
// composite kernels stage and blend float32 rows only.
__global__ void __launch_bounds__(256)
    sem_to_f32_kernel(const __nv_bfloat162* __restrict__ src, float2* __restrict__ dst, int64_t n2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __bfloat1622float2(src[i]);
}

// The Gaussian parameter arrays as (pointer, element count, bfloat16) for the
// non-finite scan, in the order reported by unigs_status_poll.
struct FiniteArrays {
    const void* ptr[7];
    int64_t count[7];
    int bf16[7];
};

// Scans array blockIdx.y for NaN and infinity (grid-stride over its
// elements); the first array found is recorded with UNIGS_ERR_NONFINITE.
__global__ void __launch_bounds__(256)
    finite_check_kernel(const FiniteArrays A, WsHeader* __restrict__ hdr) {
    const int a = blockIdx.y;
    const int64_t n = A.count[a];
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = A.bf16[a] ? __bfloat162float(static_cast<const __nv_bfloat16*>(A.ptr[a])[i])
                                  : static_cast<const float*>(A.ptr[a])[i];
        bad |= !isfinite(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        if (atomicCAS(&hdr->status, 0u, (uint32_t)UNIGS_ERR_NONFINITE) == 0u)
            hdr->nonfinite = (uint32_t)a;
    }
}

int launch_preprocess(const unigs_plan& p, const unigs_gaussians& g, const CamTable& tab,
                      void* ws, cudaStream_t st) {
    init_kernel<<<1, UNIGS_MAX_CAMS, 0, st>>>(tab, p.n_cams, ws_ptr<CamTable>(ws, p, OFF_CAM),
                                              ws_ptr<WsHeader>(ws, p, OFF_HDR));
    const int64_t total = p.n * (int64_t)p.n_cams;
    int launches = 1;
    if ((p.cfg.flags & UNIGS_FLAG_CHECK_FINITE) && p.n > 0) {
        const int64_t n = p.n, n_sh = (int64_t)(p.sh_degree + 1) * (p.sh_degree + 1);
        FiniteArrays A;
        const void* ptrs[7] = {g.mean, g.quat, g.scale, g.opacity, g.kfac, g.sh, g.sem};
        const int64_t counts[7] = {3 * n, 4 * n, 3 * n, n, n, n * n_sh * 3,
                                   p.n_sem > 0 ? n * p.n_sem : 0};
        for (int a = 0; a < 7; ++a) {
            A.ptr[a] = ptrs[a];
            A.count[a] = counts[a];
            A.bf16[a] = (a >= 5 && p.feat_dtype) ? 1 : 0;
        }
        int64_t blocks = (n * 3 + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        finite_check_kernel<<<dim3((unsigned)blocks, 7), 256, 0, st>>>(
            A, ws_ptr<WsHeader>(ws, p, OFF_HDR));
        ++launches;
    }
    if (total > 0) {
        // the list of pairs with a kept tile lives in the scan-offset region,
        // which the binning overwrites afterwards (plan_init bounds the pair
        // count below 2^32, so a pair index fits 32 bits)
        uint32_t* kept_list = ws_ptr<uint32_t>(ws, p, OFF_OFFS);
        WsHeader* hdr = ws_ptr<WsHeader>(ws, p, OFF_HDR);
        const int64_t blocks = (total + 255) / 256;
        const int64_t cap = (int64_t)sm_count() * 64;
        const int grid = (int)(blocks < cap ? blocks : cap);
        preprocess_kernel<<<grid, 256, 0, st>>>(
            g, ws_ptr<CamTable>(ws, p, OFF_CAM), p.n_cams, p.cfg.tile_w, p.cfg.tile_h,
            p.cfg.lowpass, ws_ptr<uint2>(ws, p, OFF_RECT), ws_ptr<uint32_t>(ws, p, OFF_TOUCH),
            ws_ptr<uint32_t>(ws, p, OFF_ZBITS), ws_ptr<float>(ws, p, OFF_CULL), hdr, kept_list);
        // grid-stride over the list, whose length only the device knows
        const int64_t cap2 = (int64_t)sm_count() * 32;
        const int grid2 = (int)(blocks < cap2 ? blocks : cap2);
        preprocess_splat_kernel<<<grid2, 256, 0, st>>>(
            g, ws_ptr<CamTable>(ws, p, OFF_CAM), p.cfg.lowpass, kept_list, hdr,
            ws_ptr<float>(ws, p, OFF_CULL), ws_ptr<float>(ws, p, OFF_REC),
            ws_ptr<float4>(ws, p, OFF_VP));
        launches += 2;
    }
    if (sem32_needed(p)) {
        // n * n_sem is even whenever n_sem is (rows of 2-element pairs); an odd
        // count leaves the last element to a one-element tail launch
        const int64_t cnt = p.n * (int64_t)p.n_sem;
        const int64_t n2 = cnt / 2;
        float* dst = ws_ptr<float>(ws, p, OFF_SEM32);
        if (n2 > 0) {
            const int64_t blocks = (n2 + 255) / 256;
            const int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
            sem_to_f32_kernel<<<grid, 256, 0, st>>>(
                reinterpret_cast<const __nv_bfloat162*>(g.sem), reinterpret_cast<float2*>(dst), n2);
            ++launches;
        }
        if (cnt & 1) {
            // odd total: convert the last element with a one-thread launch
            sem_tail_kernel<<<1, 1, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(g.sem) + cnt - 1,
                                             dst + cnt - 1);
            ++launches;
        }
    }
    return launches;
}

}  // namespace unigs
