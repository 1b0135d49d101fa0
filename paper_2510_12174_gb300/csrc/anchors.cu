// Anchor attribute prediction (Sec. 3.1, Fig. 2 (a)): the MLPs that turn each
// anchor into its M Gaussians, forward and backward.  The definitions are in
// include/unigs_anchors.h.
//
// The five two-layer MLPs (F = H = 32) are tiny next to the rasterizer: about
// 11 k multiply-adds per anchor, so one thread per anchor with every weight in
// shared memory (broadcast reads) is the design, not the tensor cores.
//
// Backward: each thread recomputes its anchor's hidden layers and forms the
// gradients of the MLP outputs from the decoded Gaussians' gradients; the
// per-anchor gradients (position, scale, offsets, feature, base logits, base
// k) are written by that thread.  The parameter gradients dL/dW2 = sum_a gy_a
// (x) h_a, dL/dW1 = sum_a gpre_a (x) f_a are products over the block's 128
// anchors, formed from shared-memory tiles by a fixed thread per entry and
// accumulated in shared memory across the block's grid-stride iterations;
// one float32 atomic per parameter and block adds them at the end.
#include <cuda_bf16.h>

#include "launch.h"
#include "unigs_anchors.h"
#include "unigs_internal.cuh"

namespace unigs {
namespace {

constexpr int AF = UNIGS_ANCHOR_FEAT;
constexpr int AH = UNIGS_ANCHOR_HIDDEN;
constexpr int ATHREADS = 128;
constexpr int NMLP = 5;  // sem, k, opacity, color, cov
constexpr int MAXOUT = 7 * UNIGS_ANCHOR_MAX_OFFSETS > UNIGS_MAX_SEM ? 7 * UNIGS_ANCHOR_MAX_OFFSETS
                                                                    : UNIGS_MAX_SEM;
constexpr float Y00 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))

// Offsets (in floats) of each MLP's parameters in the shared-memory block.
struct WLayout {
    int w1[NMLP], b1[NMLP], w2[NMLP], b2[NMLP], out[NMLP];
    int total;
};

struct AnchorIn {
    int64_t n;
    int M, C;
    const float *pos, *scale, *offsets, *feat, *sem, *kfac;
    const float* w1[NMLP];
    const float* b1[NMLP];
    const float* w2[NMLP];
    const float* b2[NMLP];
};

struct DecodeOut {
    float *mean, *quat, *scale, *opacity, *kfac;
    void *sh, *sem;
};

__device__ __forceinline__ float sigm(float y) { return 1.f / (1.f + expf(-y)); }

__device__ __forceinline__ void put_feat(void* base, int64_t i, float v, bool bf16) {
    if (bf16)
        static_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16_rn(v);
    else
        static_cast<float*>(base)[i] = v;
}

// Copies every MLP's parameters into shared memory (the whole block).
__device__ void load_weights(const AnchorIn& P, const WLayout& L, float* sw) {
    for (int X = 0; X < NMLP; ++X) {
        if (L.out[X] == 0) continue;
        for (int i = threadIdx.x; i < AH * AF; i += blockDim.x) sw[L.w1[X] + i] = P.w1[X][i];
        for (int i = threadIdx.x; i < AH; i += blockDim.x) sw[L.b1[X] + i] = P.b1[X][i];
        for (int i = threadIdx.x; i < L.out[X] * AH; i += blockDim.x) sw[L.w2[X] + i] = P.w2[X][i];
        for (int i = threadIdx.x; i < L.out[X]; i += blockDim.x) sw[L.b2[X] + i] = P.b2[X][i];
    }
}

// h = relu(W1 f + b1); *mask gets bit k set where the pre-activation of
// hidden unit k is positive.
__device__ __forceinline__ void hidden_layer(const float* sw, const WLayout& L, int X,
                                             const float (&f)[AF], float (&h)[AH],
                                             uint32_t* mask) {
    const float* w1 = sw + L.w1[X];
    const float* b1 = sw + L.b1[X];
    uint32_t m = 0u;
#pragma unroll
    for (int k = 0; k < AH; ++k) {
        float acc = b1[k];
#pragma unroll
        for (int i = 0; i < AF; ++i) acc = fmaf(w1[k * AF + i], f[i], acc);
        h[k] = fmaxf(acc, 0.f);
        m |= (acc > 0.f ? 1u : 0u) << k;
    }
    *mask = m;
}

// Output j of MLP X: (W2 h + b2)_j.
__device__ __forceinline__ float mlp_out(const float* sw, const WLayout& L, int X,
                                         const float (&h)[AH], int j) {
    const float* w2 = sw + L.w2[X] + j * AH;
    float acc = sw[L.b2[X] + j];
#pragma unroll
    for (int k = 0; k < AH; ++k) acc = fmaf(w2[k], h[k], acc);
    return acc;
}

__device__ __forceinline__ void load_feat(const AnchorIn& P, int64_t a, float (&f)[AF]) {
    const float4* src = reinterpret_cast<const float4*>(P.feat + a * AF);
#pragma unroll
    for (int q = 0; q < AF / 4; ++q) {
        const float4 v = src[q];
        f[4 * q] = v.x;
        f[4 * q + 1] = v.y;
        f[4 * q + 2] = v.z;
        f[4 * q + 3] = v.w;
    }
}

// The five branches run in a loop that is not unrolled, so the kernel holds
// one copy of the fully unrolled 32 x 32 hidden layer (five copies made the
// translation unit take minutes to compile).
__global__ void __launch_bounds__(ATHREADS) anchor_decode_kernel(const AnchorIn P, const WLayout L,
                                                                 const DecodeOut O, int bf16) {
    extern __shared__ __align__(16) float sw[];
    load_weights(P, L, sw);
    __syncthreads();
    const int M = P.M, C = P.C;
    const int64_t N = P.n * M;
    const bool fb = bf16 != 0;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < P.n;
         a += (int64_t)gridDim.x * blockDim.x) {
        float f[AF], h[AH];
        uint32_t mask;
        load_feat(P, a, f);
        const int64_t g0 = a * M;
        const float l[3] = {P.scale[a], P.scale[P.n + a], P.scale[2 * P.n + a]};
#pragma unroll 1
        for (int X = 0; X < NMLP; ++X) {
            if (L.out[X] == 0) continue;  // no semantic branch without logits
            hidden_layer(sw, L, X, f, h, &mask);
            if (X == 0) {
                // semantic logits: o_ah (x) sigma(MLP_sem(f)), the same for every child
                for (int c = 0; c < C; ++c) {
                    const float o = P.sem[a * C + c] * sigm(mlp_out(sw, L, 0, h, c));
                    for (int m = 0; m < M; ++m) put_feat(O.sem, (g0 + m) * C + c, o, fb);
                }
            } else if (X == 1) {
                // gradient factor: k_ah sigma(MLP_k(f))
                const float k = P.kfac[a] * sigm(mlp_out(sw, L, 1, h, 0));
                for (int m = 0; m < M; ++m) O.kfac[g0 + m] = k;
            } else if (X == 2) {
                for (int m = 0; m < M; ++m) O.opacity[g0 + m] = sigm(mlp_out(sw, L, 2, h, m));
            } else if (X == 3) {
                // colour as the degree-0 SH coefficient
                for (int m = 0; m < M; ++m)
                    for (int ch = 0; ch < 3; ++ch) {
                        const float c = sigm(mlp_out(sw, L, 3, h, 3 * m + ch));
                        put_feat(O.sh, (g0 + m) * 3 + ch, (c - 0.5f) / Y00, fb);
                    }
            } else {
                // scale and rotation
                for (int m = 0; m < M; ++m) {
                    const int64_t g = g0 + m;
                    for (int i = 0; i < 3; ++i)
                        O.scale[i * N + g] = l[i] * sigm(mlp_out(sw, L, 4, h, 7 * m + i));
                    for (int j = 0; j < 4; ++j)
                        O.quat[j * N + g] = mlp_out(sw, L, 4, h, 7 * m + 3 + j);
                }
            }
        }
        // position: x + l (x) O_m
        const float x[3] = {P.pos[a], P.pos[P.n + a], P.pos[2 * P.n + a]};
        for (int m = 0; m < M; ++m)
            for (int i = 0; i < 3; ++i)
                O.mean[i * N + g0 + m] = fmaf(l[i], P.offsets[(g0 + m) * 3 + i], x[i]);
    }
}

// ------------------------------------------------------------------ backward
struct GradIn {
    const float *mean, *quat, *scale, *opacity, *kfac, *sh, *sem;
};

struct AnchorGradOut {
    float *pos, *scale, *offsets, *feat, *sem, *kfac;
    float* w1[NMLP];
    float* b1[NMLP];
    float* w2[NMLP];
    float* b2[NMLP];
    int accumulate;
};

// Row strides (floats) of the shared-memory tiles: odd, so that the rows of
// a warp's 32 threads start in 32 different banks.
constexpr int GYS = MAXOUT + 1;
constexpr int HS = AH + 1;
constexpr int FS = AF + 1;

__host__ __device__ constexpr size_t bwd_tile_floats() {
    return (size_t)ATHREADS * (GYS + 2 * HS + FS);
}

__device__ __forceinline__ float gin(const float* p, int64_t i) { return p ? p[i] : 0.f; }
__device__ __forceinline__ void put(float* p, int64_t i, float v, int acc) {
    if (acc)
        p[i] += v;
    else
        p[i] = v;
}

__global__ void __launch_bounds__(ATHREADS) anchor_decode_bwd_kernel(const AnchorIn P,
                                                                     const WLayout L,
                                                                     const GradIn G,
                                                                     const AnchorGradOut R) {
    extern __shared__ __align__(16) float sm[];
    float* sw = sm;                     // parameters
    float* sg = sw + L.total;           // parameter gradients of this block
    float* gy = sg + L.total;           // [ATHREADS][GYS] output gradients of one branch
    float* hid = gy + ATHREADS * GYS;   // [ATHREADS][HS] hidden activations
    float* gpre = hid + ATHREADS * HS;  // [ATHREADS][HS] pre-activation gradients
    float* ft = gpre + ATHREADS * HS;   // [ATHREADS][FS] features
    load_weights(P, L, sw);
    for (int i = threadIdx.x; i < L.total; i += blockDim.x) sg[i] = 0.f;
    __syncthreads();
    const int tid = threadIdx.x, M = P.M, C = P.C, acc = R.accumulate;
    const int64_t N = P.n * M;
    for (int64_t base = blockIdx.x * (int64_t)ATHREADS; base < P.n;
         base += (int64_t)gridDim.x * ATHREADS) {
        const int64_t a = base + tid;
        const bool valid = a < P.n;
        const int rows = (int)min((int64_t)ATHREADS, P.n - base);
        const int64_t g0 = a * M;
        float f[AF], gf[AF];
        if (valid)
            load_feat(P, a, f);
        else
#pragma unroll
            for (int i = 0; i < AF; ++i) f[i] = 0.f;
#pragma unroll
        for (int i = 0; i < AF; ++i) {
            ft[tid * FS + i] = f[i];
            gf[i] = 0.f;
        }
        float l[3] = {0.f, 0.f, 0.f}, gl[3] = {0.f, 0.f, 0.f};
        if (valid)
            for (int i = 0; i < 3; ++i) l[i] = P.scale[i * P.n + a];
        float* gyr = gy + tid * GYS;
        for (int X = 0; X < NMLP; ++X) {
            const int out = L.out[X];
            if (out == 0) continue;  // uniform: no semantic branch without logits
            float h[AH];
            uint32_t mask;
            hidden_layer(sw, L, X, f, h, &mask);
            // dL/d(branch output)
            if (!valid) {
                for (int j = 0; j < out; ++j) gyr[j] = 0.f;
            } else if (X == 0) {
                for (int c = 0; c < C; ++c) {
                    const float s = sigm(mlp_out(sw, L, 0, h, c));
                    float gc = 0.f;
                    for (int m = 0; m < M; ++m) gc += gin(G.sem, (g0 + m) * C + c);
                    put(R.sem, a * C + c, gc * s, acc);
                    gyr[c] = gc * P.sem[a * C + c] * s * (1.f - s);
                }
            } else if (X == 1) {
                const float s = sigm(mlp_out(sw, L, 1, h, 0));
                float gk = 0.f;
                for (int m = 0; m < M; ++m) gk += gin(G.kfac, g0 + m);
                put(R.kfac, a, gk * s, acc);
                gyr[0] = gk * P.kfac[a] * s * (1.f - s);
            } else if (X == 2) {
                for (int m = 0; m < M; ++m) {
                    const float s = sigm(mlp_out(sw, L, 2, h, m));
                    gyr[m] = gin(G.opacity, g0 + m) * s * (1.f - s);
                }
            } else if (X == 3) {
                for (int j = 0; j < 3 * M; ++j) {
                    const float c = sigm(mlp_out(sw, L, 3, h, j));
                    gyr[j] = gin(G.sh, g0 * 3 + j) / Y00 * c * (1.f - c);
                }
            } else {
                for (int m = 0; m < M; ++m) {
                    const int64_t g = g0 + m;
                    for (int i = 0; i < 3; ++i) {
                        const float s = sigm(mlp_out(sw, L, 4, h, 7 * m + i));
                        const float gs = gin(G.scale, i * N + g);
                        gyr[7 * m + i] = gs * l[i] * s * (1.f - s);
                        gl[i] = fmaf(gs, s, gl[i]);
                    }
                    for (int j = 0; j < 4; ++j) gyr[7 * m + 3 + j] = gin(G.quat, j * N + g);
                }
            }
#pragma unroll
            for (int k = 0; k < AH; ++k) hid[tid * HS + k] = h[k];
            // back through the branch: dL/dh = W2^T gy, the relu, dL/df += W1^T gpre
            float gh[AH];
#pragma unroll
            for (int k = 0; k < AH; ++k) gh[k] = 0.f;
            for (int j = 0; j < out; ++j) {
                const float v = gyr[j];
                const float* w2 = sw + L.w2[X] + j * AH;
#pragma unroll
                for (int k = 0; k < AH; ++k) gh[k] = fmaf(w2[k], v, gh[k]);
            }
            const float* w1 = sw + L.w1[X];
#pragma unroll
            for (int k = 0; k < AH; ++k) {
                const float gp = ((mask >> k) & 1u) ? gh[k] : 0.f;
                gpre[tid * HS + k] = gp;
#pragma unroll
                for (int i = 0; i < AF; ++i) gf[i] = fmaf(w1[k * AF + i], gp, gf[i]);
            }
            __syncthreads();
            // parameter gradients over the block's anchors; every entry has a
            // fixed owner thread, so the shared accumulators need no atomics
            for (int e = tid; e < out * AH; e += ATHREADS) {
                const int j = e / AH, k = e % AH;
                float s = 0.f;
                for (int r = 0; r < rows; ++r) s = fmaf(gy[r * GYS + j], hid[r * HS + k], s);
                sg[L.w2[X] + e] += s;
            }
            for (int j = tid; j < out; j += ATHREADS) {
                float s = 0.f;
                for (int r = 0; r < rows; ++r) s += gy[r * GYS + j];
                sg[L.b2[X] + j] += s;
            }
            for (int e = tid; e < AH * AF; e += ATHREADS) {
                const int k = e / AF, i = e % AF;
                float s = 0.f;
                for (int r = 0; r < rows; ++r) s = fmaf(gpre[r * HS + k], ft[r * FS + i], s);
                sg[L.w1[X] + e] += s;
            }
            for (int k = tid; k < AH; k += ATHREADS) {
                float s = 0.f;
                for (int r = 0; r < rows; ++r) s += gpre[r * HS + k];
                sg[L.b1[X] + k] += s;
            }
            __syncthreads();
        }
        if (valid) {
            // position and offsets: mu_m = x + l (x) O_m
            float gx[3] = {0.f, 0.f, 0.f};
            for (int m = 0; m < M; ++m)
                for (int i = 0; i < 3; ++i) {
                    const float gm = gin(G.mean, i * N + g0 + m);
                    gx[i] += gm;
                    gl[i] = fmaf(gm, P.offsets[(g0 + m) * 3 + i], gl[i]);
                    put(R.offsets, (g0 + m) * 3 + i, gm * l[i], acc);
                }
            for (int i = 0; i < 3; ++i) {
                put(R.pos, i * P.n + a, gx[i], acc);
                put(R.scale, i * P.n + a, gl[i], acc);
            }
#pragma unroll
            for (int i = 0; i < AF; ++i) put(R.feat, a * AF + i, gf[i], acc);
        }
    }
    // one atomic per parameter and block (cleared by the host without accumulate)
    for (int X = 0; X < NMLP; ++X) {
        if (L.out[X] == 0) continue;
        for (int i = threadIdx.x; i < AH * AF; i += blockDim.x)
            atomicAdd(R.w1[X] + i, sg[L.w1[X] + i]);
        for (int i = threadIdx.x; i < AH; i += blockDim.x) atomicAdd(R.b1[X] + i, sg[L.b1[X] + i]);
        for (int i = threadIdx.x; i < L.out[X] * AH; i += blockDim.x)
            atomicAdd(R.w2[X] + i, sg[L.w2[X] + i]);
        for (int i = threadIdx.x; i < L.out[X]; i += blockDim.x)
            atomicAdd(R.b2[X] + i, sg[L.b2[X] + i]);
    }
}

}  // namespace
}  // namespace unigs

// ------------------------------------------------------------------ C ABI
namespace {

using unigs::AH;
using unigs::AF;
using unigs::NMLP;

bool mlp_ok(const unigs_mlp& m) { return m.w1 && m.b1 && m.w2 && m.b2; }
bool mlp_ok(const unigs_mlp_grads& m) { return m.w1 && m.b1 && m.w2 && m.b2; }

bool anchors_ok(const unigs_anchors* a) {
    if (!a || a->n < 0 || a->n_offsets < 1 || a->n_offsets > UNIGS_ANCHOR_MAX_OFFSETS ||
        a->feat_dim != UNIGS_ANCHOR_FEAT || a->hidden != UNIGS_ANCHOR_HIDDEN || a->n_sem < 0 ||
        a->n_sem > UNIGS_MAX_SEM)
        return false;
    if (a->n == 0) return true;
    if (!a->pos || !a->scale || !a->offsets || !a->feat || !a->kfac) return false;
    if (reinterpret_cast<uintptr_t>(a->feat) & 15) return false;
    if (a->n_sem > 0 && (!a->sem || !mlp_ok(a->mlp_sem))) return false;
    return mlp_ok(a->mlp_k) && mlp_ok(a->mlp_opacity) && mlp_ok(a->mlp_color) &&
           mlp_ok(a->mlp_cov);
}

void make_layout(const unigs_anchors& a, unigs::WLayout& L, unigs::AnchorIn& P) {
    const int M = a.n_offsets;
    const int outs[NMLP] = {a.n_sem, 1, M, 3 * M, 7 * M};
    const unigs_mlp* mlps[NMLP] = {&a.mlp_sem, &a.mlp_k, &a.mlp_opacity, &a.mlp_color, &a.mlp_cov};
    int off = 0;
    for (int X = 0; X < NMLP; ++X) {
        L.out[X] = outs[X];
        P.w1[X] = mlps[X]->w1;
        P.b1[X] = mlps[X]->b1;
        P.w2[X] = mlps[X]->w2;
        P.b2[X] = mlps[X]->b2;
        L.w1[X] = L.b1[X] = L.w2[X] = L.b2[X] = off;
        if (outs[X] == 0) continue;
        L.w1[X] = off;
        off += AH * AF;
        L.b1[X] = off;
        off += AH;
        L.w2[X] = off;
        off += outs[X] * AH;
        L.b2[X] = off;
        off += outs[X];
    }
    L.total = off;
    P.n = a.n;
    P.M = M;
    P.C = a.n_sem;
    P.pos = a.pos;
    P.scale = a.scale;
    P.offsets = a.offsets;
    P.feat = a.feat;
    P.sem = a.sem;
    P.kfac = a.kfac;
}

int anchor_grid(int64_t n) {
    const int64_t blocks = (n + unigs::ATHREADS - 1) / unigs::ATHREADS;
    const int64_t cap = (int64_t)unigs::sm_count() * 8;
    return (int)(blocks < cap ? blocks : cap);
}

unigs_status launch_status() {
    return cudaGetLastError() == cudaSuccess ? UNIGS_OK : UNIGS_ERR_CUDA;
}

}  // namespace

extern "C" unigs_status unigs_anchor_decode(const unigs_anchors* a,
                                            const unigs_anchor_gaussians* out,
                                            unigs_stream stream) {
    if (!anchors_ok(a) || !out || (out->feat_dtype != 0 && out->feat_dtype != 1))
        return UNIGS_ERR_INVALID_ARG;
    if (a->n == 0) return UNIGS_OK;
    if (!out->mean || !out->quat || !out->scale || !out->opacity || !out->kfac || !out->sh ||
        (a->n_sem > 0 && !out->sem))
        return UNIGS_ERR_INVALID_ARG;
    unigs::WLayout L;
    unigs::AnchorIn P;
    make_layout(*a, L, P);
    unigs::DecodeOut O{out->mean, out->quat, out->scale, out->opacity, out->kfac, out->sh,
                       out->sem};
    const size_t smem = sizeof(float) * (size_t)L.total;
    const int grid = anchor_grid(a->n);
    cudaStream_t st = (cudaStream_t)stream;
    unigs::ensure_smem_limit(reinterpret_cast<const void*>(&unigs::anchor_decode_kernel), (int)smem);
    unigs::anchor_decode_kernel<<<grid, unigs::ATHREADS, smem, st>>>(P, L, O, out->feat_dtype);
    return launch_status();
}

extern "C" unigs_status unigs_anchor_decode_bwd(const unigs_anchors* a, const unigs_param_grads* g,
                                                const unigs_anchor_grads* out,
                                                unigs_stream stream) {
    if (!anchors_ok(a) || !g || !out) return UNIGS_ERR_INVALID_ARG;
    if (!out->pos || !out->scale || !out->offsets || !out->feat || !out->kfac ||
        (a->n_sem > 0 && (!out->sem || !mlp_ok(out->mlp_sem))) || !mlp_ok(out->mlp_k) ||
        !mlp_ok(out->mlp_opacity) || !mlp_ok(out->mlp_color) || !mlp_ok(out->mlp_cov))
        return UNIGS_ERR_INVALID_ARG;
    unigs::WLayout L;
    unigs::AnchorIn P;
    make_layout(*a, L, P);
    cudaStream_t st = (cudaStream_t)stream;
    const unigs_mlp_grads* mg[NMLP] = {&out->mlp_sem, &out->mlp_k, &out->mlp_opacity,
                                       &out->mlp_color, &out->mlp_cov};
    unigs::AnchorGradOut R;
    R.pos = out->pos;
    R.scale = out->scale;
    R.offsets = out->offsets;
    R.feat = out->feat;
    R.sem = out->sem;
    R.kfac = out->kfac;
    R.accumulate = out->accumulate ? 1 : 0;
    for (int X = 0; X < NMLP; ++X) {
        R.w1[X] = mg[X]->w1;
        R.b1[X] = mg[X]->b1;
        R.w2[X] = mg[X]->w2;
        R.b2[X] = mg[X]->b2;
        if (L.out[X] == 0 || out->accumulate) continue;
        // the parameter gradients are sums of atomics: cleared first
        cudaMemsetAsync(R.w1[X], 0, sizeof(float) * AH * AF, st);
        cudaMemsetAsync(R.b1[X], 0, sizeof(float) * AH, st);
        cudaMemsetAsync(R.w2[X], 0, sizeof(float) * L.out[X] * AH, st);
        cudaMemsetAsync(R.b2[X], 0, sizeof(float) * L.out[X], st);
    }
    if (a->n == 0) return launch_status();
    unigs::GradIn G{g->mean, g->quat, g->scale, g->opacity, g->kfac, g->sh, g->sem};
    const size_t smem = sizeof(float) * (2 * (size_t)L.total + unigs::bwd_tile_floats());
    const int64_t blocks = (a->n + unigs::ATHREADS - 1) / unigs::ATHREADS;
    const int grid = (int)(blocks < unigs::sm_count() ? blocks : unigs::sm_count());
    unigs::ensure_smem_limit(reinterpret_cast<const void*>(&unigs::anchor_decode_bwd_kernel),
                             (int)smem);
    unigs::anchor_decode_bwd_kernel<<<grid, unigs::ATHREADS, smem, st>>>(P, L, G, R);
    return launch_status();
}
