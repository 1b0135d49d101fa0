// Normal from depth (Alg. 1) and its backward (Alg. 3).
//
// The back-projection of the supplement's Sec. 3, P_world = R_cw (d~ D) + C
// with d~ = ((u-cx)/fx, (v-cy)/fy, 1), is evaluated in the camera frame: the
// centre C cancels in every central difference, and the cross product
// commutes with the rotation, so n_world = R_cw n_cam.  A difference of two
// back-projected points along x is written
//   P(u+g) - P(u-g) = (x~(u+g) (D+ - D-) + (2g/fx) D-, y~ (D+ - D-), D+ - D-)
// so that no large, nearly equal coordinates are subtracted.  The view
// correction flips the normal when it points away from the camera, i.e. when
// n_cam . P_cam > 0 (P_world - C = R_cw P_cam).
//
// The backward is a gather: each pixel sums, over the stencils of its
// neighbours that use it, d(loss)/d(point) dotted with d~ (the derivative of
// the back-projected point w.r.t. the depth).  The paper scatters the same
// terms with atomics; the gather is deterministic.
#include "launch.h"

namespace unigs {

constexpr int MAX_STEP = 4;

// The normal-from-depth kernels work on blocks of DN_TILE x DN_TILE pixels
// of their own (independent of the binning tile shape): block b of the launch
// belongs to the camera k with blk_off[k] <= b < blk_off[k + 1] and is block
// b - blk_off[k] of that camera, row-major with blk_x[k] blocks per row.
constexpr int DN_TILE = 16;

struct DNParams {
    CamTable tab;  // by value: these entry points take no workspace
    int32_t blk_off[UNIGS_MAX_CAMS + 1];
    int32_t blk_x[UNIGS_MAX_CAMS];
    int n_cams;
    int step1, step2;
    float lambda;
    const float* depth;
    float* normal_d;
    const float* g_normal;
    const float* g_depth_in;
    float* g_depth_out;
};

// The camera whose blocks contain blockIdx.x.
__device__ __forceinline__ void dn_block(const DNParams& P, int* k) {
    int c = 0;
    for (int j = 1; j < P.n_cams; ++j)
        if ((int)blockIdx.x >= P.blk_off[j]) c = j;
    *k = c;
}

// Camera-frame difference of two back-projected points along x or y.
__device__ __forceinline__ void diff_x(float xt_p, float yt, float Dp, float Dm, float two_g_fx,
                                       float* v) {
    const float dD = Dp - Dm;
    v[0] = fmaf(xt_p, dD, two_g_fx * Dm);
    v[1] = yt * dD;
    v[2] = dD;
}
__device__ __forceinline__ void diff_y(float xt, float yt_p, float Dp, float Dm, float two_g_fy,
                                       float* v) {
    const float dD = Dp - Dm;
    v[0] = xt * dD;
    v[1] = fmaf(yt_p, dD, two_g_fy * Dm);
    v[2] = dD;
}
__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Forward state of one pixel from a depth accessor D(du, dv) (offsets from
// the pixel).  Returns false when the stencil leaves the image or the fused
// vector is zero.
struct DNState {
    float vx[2][3], vy[2][3], n[2][3], sgn, nf[3], norm, N[3];
    bool flip;
};

template <typename DF>
__device__ __forceinline__ bool dn_forward(const DevCam& cam, int u, int v, int step1, int step2,
                                           float lambda, DF D, DNState& s) {
    const int smax = max(step1, step2);
    if (u - smax < 0 || v - smax < 0 || u + smax >= cam.width || v + smax >= cam.height)
        return false;
    const float xt = ((float)u - cam.cx) / cam.fx, yt = ((float)v - cam.cy) / cam.fy;
    const int steps[2] = {step1, step2};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int g = steps[k];
        const float xtp = ((float)(u + g) - cam.cx) / cam.fx;
        const float ytp = ((float)(v + g) - cam.cy) / cam.fy;
        diff_x(xtp, yt, D(g, 0), D(-g, 0), (2.f * g) / cam.fx, s.vx[k]);
        diff_y(xt, ytp, D(0, g), D(0, -g), (2.f * g) / cam.fy, s.vy[k]);
        cross3(s.vx[k], s.vy[k], s.n[k]);
    }
    const float d12 = s.n[0][0] * s.n[1][0] + s.n[0][1] * s.n[1][1] + s.n[0][2] * s.n[1][2];
    s.sgn = d12 >= 0.f ? 1.f : -1.f;
    const float l1 = lambda, l2 = (1.f - lambda) * s.sgn;
#pragma unroll
    for (int i = 0; i < 3; ++i) s.nf[i] = fmaf(l1, s.n[0][i], l2 * s.n[1][i]);
    s.norm = sqrtf(s.nf[0] * s.nf[0] + s.nf[1] * s.nf[1] + s.nf[2] * s.nf[2]);
    if (!(s.norm > 0.f)) return false;
    const float inv = 1.f / s.norm;
#pragma unroll
    for (int i = 0; i < 3; ++i) s.N[i] = s.nf[i] * inv;
    const float D0 = D(0, 0);
    const float dp = (s.N[0] * xt + s.N[1] * yt + s.N[2]) * D0;  // N . P_cam
    s.flip = dp > 0.f;
    return true;
}

__global__ void __launch_bounds__(256) depth_normal_fwd_kernel(const __grid_constant__ DNParams P) {
    int k = 0;
    dn_block(P, &k);
    const DevCam& cam = P.tab.cam[k];
    const int lt = (int)blockIdx.x - P.blk_off[k];
    const int u = (lt % P.blk_x[k]) * DN_TILE + (threadIdx.x & 15);
    const int v = (lt / P.blk_x[k]) * DN_TILE + (threadIdx.x >> 4);
    if (u >= cam.width || v >= cam.height) return;
    const int W = cam.width;
    const int64_t HW = (int64_t)cam.height * W;
    const float* Dimg = P.depth + cam.pix_off;
    auto D = [&](int du, int dv) { return __ldg(Dimg + (int64_t)(v + dv) * W + (u + du)); };
    DNState s;
    float out[3] = {0.f, 0.f, 0.f};
    if (dn_forward(cam, u, v, P.step1, P.step2, P.lambda, D, s)) {
        const float sg = s.flip ? -1.f : 1.f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            out[i] = sg * (cam.R_cw[3 * i] * s.N[0] + cam.R_cw[3 * i + 1] * s.N[1] +
                           cam.R_cw[3 * i + 2] * s.N[2]);
    }
    const int64_t idx = (int64_t)v * W + u;
    float* o = P.normal_d + cam.pix_off * 3;
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i * HW + idx] = out[i];
}

// Backward.  Shared memory: the depth tile with a halo of 2*smax, and for every
// pixel q of the tile plus a halo of smax the gradients w.r.t. its four
// difference vectors (vx1, vy1, vx2, vy2), camera frame.
__global__ void __launch_bounds__(256) depth_normal_bwd_kernel(const __grid_constant__ DNParams P) {
    constexpr int DP_MAX = DN_TILE + 4 * MAX_STEP;  // depth tile pitch
    constexpr int GP_MAX = DN_TILE + 2 * MAX_STEP;  // gradient tile pitch
    __shared__ float sD[DP_MAX * DP_MAX];
    __shared__ float sG[GP_MAX * GP_MAX][12];
    int k = 0;
    dn_block(P, &k);
    const DevCam& cam = P.tab.cam[k];
    const int lt = (int)blockIdx.x - P.blk_off[k];
    const int u0 = (lt % P.blk_x[k]) * DN_TILE, v0 = (lt / P.blk_x[k]) * DN_TILE;
    const int W = cam.width, H = cam.height;
    const int64_t HW = (int64_t)H * W;
    const int h = max(P.step1, P.step2);
    const int dp = DN_TILE + 4 * h, gp = DN_TILE + 2 * h;
    const float* Dimg = P.depth + cam.pix_off;
    const float* gN = P.g_normal + cam.pix_off * 3;

    for (int j = threadIdx.x; j < dp * dp; j += blockDim.x) {
        const int uu = u0 - 2 * h + j % dp, vv = v0 - 2 * h + j / dp;
        sD[j] = (uu >= 0 && vv >= 0 && uu < W && vv < H) ? __ldg(Dimg + (int64_t)vv * W + uu) : 0.f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < gp * gp; j += blockDim.x) {
        const int qu = u0 - h + j % gp, qv = v0 - h + j / gp;
        float gv[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) gv[k] = 0.f;
        if (qu >= 0 && qv >= 0 && qu < W && qv < H) {
            const int cu = qu - (u0 - 2 * h), cv = qv - (v0 - 2 * h);
            auto D = [&](int du, int dv) { return sD[(cv + dv) * dp + (cu + du)]; };
            DNState s;
            if (dn_forward(cam, qu, qv, P.step1, P.step2, P.lambda, D, s)) {
                const int64_t qi = (int64_t)qv * W + qu;
                const float gw[3] = {__ldg(gN + qi), __ldg(gN + HW + qi), __ldg(gN + 2 * HW + qi)};
                // world -> camera frame (transpose of R_cw), undo the flip
                const float sg = s.flip ? -1.f : 1.f;
                float g[3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    g[i] = sg * (cam.R_cw[i] * gw[0] + cam.R_cw[3 + i] * gw[1] +
                                 cam.R_cw[6 + i] * gw[2]);
                // normalisation Jacobian (I - N N^T) / |n_fused|
                const float dgn = g[0] * s.N[0] + g[1] * s.N[1] + g[2] * s.N[2];
                const float inv = 1.f / s.norm;
                float gnf[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) gnf[i] = (g[i] - dgn * s.N[i]) * inv;
                // fusion weights lambda and (1 - lambda) sign(n1.n2)
                const float wk[2] = {P.lambda, (1.f - P.lambda) * s.sgn};
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float gn[3] = {wk[k] * gnf[0], wk[k] * gnf[1], wk[k] * gnf[2]};
                    // n = vx x vy:  dL/dvx = vy x gn,  dL/dvy = gn x vx
                    cross3(s.vy[k], gn, &gv[6 * k]);
                    cross3(gn, s.vx[k], &gv[6 * k + 3]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) sG[j][k] = gv[k];
    }
    __syncthreads();
    const int lu = threadIdx.x & 15, lv = threadIdx.x >> 4;
    const int u = u0 + lu, v = v0 + lv;
    if (u >= W || v >= H) return;
    float gP[3] = {0.f, 0.f, 0.f};
    const int steps[2] = {P.step1, P.step2};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int g = steps[k];
        const int cu = lu + h, cv = lv + h;  // position in the gradient tile
        const float* a = sG[cv * gp + (cu - g)] + 6 * k;      // q = p - g e_x : +dvx
        const float* b = sG[cv * gp + (cu + g)] + 6 * k;      // q = p + g e_x : -dvx
        const float* c = sG[(cv - g) * gp + cu] + 6 * k + 3;  // q = p - g e_y : +dvy
        const float* d = sG[(cv + g) * gp + cu] + 6 * k + 3;  // q = p + g e_y : -dvy
#pragma unroll
        for (int i = 0; i < 3; ++i) gP[i] += (a[i] - b[i]) + (c[i] - d[i]);
    }
    const float xt = ((float)u - cam.cx) / cam.fx, yt = ((float)v - cam.cy) / cam.fy;
    const float gD = gP[0] * xt + gP[1] * yt + gP[2];
    const int64_t idx = cam.pix_off + (int64_t)v * W + u;
    const float base = P.g_depth_in ? P.g_depth_in[idx] : 0.f;
    P.g_depth_out[idx] = base + gD;
}

static void make_dn(const unigs_plan& p, const CamTable& tab, DNParams& P) {
    P.tab = tab;
    P.n_cams = p.n_cams;
    int32_t off = 0;
    for (int k = 0; k < p.n_cams; ++k) {
        P.blk_off[k] = off;
        P.blk_x[k] = (tab.cam[k].width + DN_TILE - 1) / DN_TILE;
        off += P.blk_x[k] * ((tab.cam[k].height + DN_TILE - 1) / DN_TILE);
    }
    P.blk_off[p.n_cams] = off;
    P.step1 = p.cfg.step1;
    P.step2 = p.cfg.step2;
    P.lambda = p.cfg.lambda;
}

int launch_depth_normal_fwd(const unigs_plan& p, const CamTable& tab, const float* depth,
                            float* normal_d, cudaStream_t st) {
    if (p.n_tiles == 0) return 0;
    static thread_local DNParams P;
    make_dn(p, tab, P);
    P.depth = depth;
    P.normal_d = normal_d;
    P.g_normal = nullptr;
    P.g_depth_in = nullptr;
    P.g_depth_out = nullptr;
    depth_normal_fwd_kernel<<<(unsigned)P.blk_off[p.n_cams], 256, 0, st>>>(P);
    return 1;
}

int launch_depth_normal_bwd(const unigs_plan& p, const CamTable& tab, const float* depth,
                            const float* g_normal_d, const float* g_depth_in, float* g_depth_out,
                            cudaStream_t st) {
    if (p.n_tiles == 0) return 0;
    static thread_local DNParams P;
    make_dn(p, tab, P);
    P.depth = depth;
    P.normal_d = nullptr;
    P.g_normal = g_normal_d;
    P.g_depth_in = g_depth_in;
    P.g_depth_out = g_depth_out;
    depth_normal_bwd_kernel<<<(unsigned)P.blk_off[p.n_cams], 256, 0, st>>>(P);
    return 1;
}

}  // namespace unigs
