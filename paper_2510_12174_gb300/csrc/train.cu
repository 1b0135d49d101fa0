// Training step around the rasterizer: the combined loss of Sec. 3.4 (without
// SSIM) with its gradients, the Adam update with float32 master values and
// bfloat16 feature copies, and the k-pruning rule of Sec. 3.3.
//
// All three are streaming (HBM-bound) kernels: the loss reads each rendered
// map and target once per pass (two passes: sums, then gradients, because the
// magnitude-normalised weights depend on the whole-batch sums), Adam reads
// and writes every parameter and its moments once, and the pruning compaction
// moves every surviving parameter once.
#include "launch.h"

namespace unigs {

// ------------------------------------------------------------------ losses
constexpr int LOSS_THREADS = 256;
constexpr int LOSS_SUMS = 8;  // l1, normal dot, depth, n_depth, seg, n_label, K, unused

struct LossParams {
    int n_cams, n_sem;
    int64_t n_pixels;
    int64_t pix_off[UNIGS_MAX_CAMS + 1];
    const float* rgb;
    const float* depth;
    const float* kmap;
    const float* logits;
    const float* normal_d;
    unigs_targets tgt;
    unigs_loss_lambda lam;
    float* partial;  // [gridDim.x][LOSS_SUMS]
    float* record;
    unigs_loss_grads g;
};

// Camera of global pixel gp and the pixel's index inside that camera.
__device__ __forceinline__ void pixel_cam(const LossParams& P, int64_t gp, int* k, int64_t* idx,
                                          int64_t* hw) {
    int lo = 0, hi = P.n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.pix_off[mid] <= gp) lo = mid; else hi = mid - 1;
    }
    *k = lo;
    *idx = gp - P.pix_off[lo];
    *hw = P.pix_off[lo + 1] - P.pix_off[lo];
}

__device__ __forceinline__ float sgn(float x) { return (float)((x > 0.f) - (x < 0.f)); }

// The logits of one pixel (planar channels) into registers, padding with
// -inf, and their maximum and sum of exponentials.
template <int NS>
__device__ __forceinline__ void pixel_logits(const float* O, int64_t hw, int C, float (&o)[NS],
                                             float* mx_out, float* z_out) {
    float mx = -INFINITY;
#pragma unroll
    for (int c = 0; c < NS; ++c) {
        o[c] = c < C ? O[(int64_t)c * hw] : -INFINITY;
        mx = fmaxf(mx, o[c]);
    }
    float z = 0.f;
#pragma unroll
    for (int c = 0; c < NS; ++c)
        if (c < C) z += expf(o[c] - mx);
    *mx_out = mx;
    *z_out = z;
}

__device__ __forceinline__ float block_sum(float v, float* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;  // valid in thread 0
}

template <int NS>
__global__ void __launch_bounds__(LOSS_THREADS) loss_sums_kernel(const LossParams P) {
    __shared__ float sh[32];
    float acc[LOSS_SUMS] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < P.n_pixels;
         gp += (int64_t)gridDim.x * blockDim.x) {
        int k;
        int64_t idx, hw;
        pixel_cam(P, gp, &k, &idx, &hw);
        const int64_t po = P.pix_off[k];
        if (P.tgt.rgb)
            for (int c = 0; c < 3; ++c) {
                const int64_t e = po * 3 + c * hw + idx;
                acc[0] += fabsf(P.rgb[e] - P.tgt.rgb[e]);
            }
        if (P.tgt.normal)
            for (int c = 0; c < 3; ++c) {
                const int64_t e = po * 3 + c * hw + idx;
                acc[1] = fmaf(P.normal_d[e], P.tgt.normal[e], acc[1]);
            }
        if (P.tgt.depth) {
            const float dt = P.tgt.depth[gp];
            if (dt > 0.f) {
                acc[2] += fabsf(P.depth[gp] - dt);
                acc[3] += 1.f;
            }
        }
        if (NS > 0 && P.tgt.label) {
            const int lab = P.tgt.label[gp];
            if (lab >= 0 && lab < P.n_sem) {
                constexpr int N1 = NS > 0 ? NS : 1;
                float o[N1], mx, z;
                pixel_logits<N1>(P.logits + po * P.n_sem + idx, hw, P.n_sem, o, &mx, &z);
                float ol = 0.f;
#pragma unroll
                for (int c = 0; c < N1; ++c)
                    if (c == lab) ol = o[c];
                acc[4] += mx + logf(z) - ol;
                acc[5] += 1.f;
            }
        }
        if (P.kmap) acc[6] += fabsf(P.kmap[gp] - 1.f);
    }
    for (int s = 0; s < LOSS_SUMS; ++s) {
        const float t = block_sum(acc[s], sh);
        if (threadIdx.x == 0) P.partial[(int64_t)blockIdx.x * LOSS_SUMS + s] = t;
    }
}

// One block: sums the block partials in a fixed order, forms the terms and
// the weights (Sec. 3.4) and writes the record.
__global__ void __launch_bounds__(LOSS_THREADS) loss_finalize_kernel(const LossParams P, int nb) {
    __shared__ float sh[32];
    __shared__ float tot[LOSS_SUMS];
    for (int s = 0; s < LOSS_SUMS; ++s) {
        float v = 0.f;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) v += P.partial[(int64_t)b * LOSS_SUMS + s];
        const float t = block_sum(v, sh);
        if (threadIdx.x == 0) tot[s] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const float Pf = (float)P.n_pixels;
    const float L_l1 = P.tgt.rgb ? tot[0] / (3.f * Pf) : 0.f;
    const float L_n = P.tgt.normal ? 1.f - tot[1] / Pf : 0.f;
    const float L_d = (P.tgt.depth && tot[3] > 0.f) ? tot[2] / tot[3] : 0.f;
    const float L_s = (P.tgt.label && tot[5] > 0.f) ? tot[4] / tot[5] : 0.f;
    const float L_k = P.kmap ? tot[6] / Pf : 0.f;
    const float a = fabsf(L_l1);
    const float w_l1 = P.tgt.rgb ? P.lam.l1 : 0.f;
    const float w_n = L_n != 0.f ? P.lam.normal * a / fabsf(L_n) : 0.f;
    const float w_d = L_d != 0.f ? P.lam.depth * a / fabsf(L_d) : 0.f;
    const float w_s = L_s != 0.f ? P.lam.seg * a / fabsf(L_s) : 0.f;
    const float w_k = L_k != 0.f ? P.lam.K * a / fabsf(L_k) : 0.f;
    float* r = P.record;
    r[UNIGS_LOSS_TOTAL] = w_l1 * L_l1 + w_n * L_n + w_d * L_d + w_s * L_s + w_k * L_k;
    r[UNIGS_LOSS_L1] = L_l1;
    r[UNIGS_LOSS_NORMAL] = L_n;
    r[UNIGS_LOSS_DEPTH] = L_d;
    r[UNIGS_LOSS_SEG] = L_s;
    r[UNIGS_LOSS_K] = L_k;
    r[UNIGS_LOSS_W_L1] = w_l1;
    r[UNIGS_LOSS_W_NORMAL] = w_n;
    r[UNIGS_LOSS_W_DEPTH] = w_d;
    r[UNIGS_LOSS_W_SEG] = w_s;
    r[UNIGS_LOSS_W_K] = w_k;
    r[UNIGS_LOSS_N_DEPTH] = tot[3];
    r[UNIGS_LOSS_N_LABEL] = tot[5];
    r[13] = r[14] = r[15] = 0.f;
}

template <int NS>
__global__ void __launch_bounds__(LOSS_THREADS) loss_grad_kernel(const LossParams P) {
    const float* r = P.record;
    const float Pf = (float)P.n_pixels;
    const float a_rgb = r[UNIGS_LOSS_W_L1] / (3.f * Pf);
    const float a_n = -r[UNIGS_LOSS_W_NORMAL] / Pf;
    const float a_d = r[UNIGS_LOSS_N_DEPTH] > 0.f ? r[UNIGS_LOSS_W_DEPTH] / r[UNIGS_LOSS_N_DEPTH] : 0.f;
    const float a_s = r[UNIGS_LOSS_N_LABEL] > 0.f ? r[UNIGS_LOSS_W_SEG] / r[UNIGS_LOSS_N_LABEL] : 0.f;
    const float a_k = r[UNIGS_LOSS_W_K] / Pf;
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < P.n_pixels;
         gp += (int64_t)gridDim.x * blockDim.x) {
        int k;
        int64_t idx, hw;
        pixel_cam(P, gp, &k, &idx, &hw);
        const int64_t po = P.pix_off[k];
        if (P.g.rgb)
            for (int c = 0; c < 3; ++c) {
                const int64_t e = po * 3 + c * hw + idx;
                P.g.rgb[e] = P.tgt.rgb ? a_rgb * sgn(P.rgb[e] - P.tgt.rgb[e]) : 0.f;
            }
        if (P.g.normal_d)
            for (int c = 0; c < 3; ++c) {
                const int64_t e = po * 3 + c * hw + idx;
                P.g.normal_d[e] = P.tgt.normal ? a_n * P.tgt.normal[e] : 0.f;
            }
        if (P.g.depth) {
            float g = 0.f;
            if (P.tgt.depth) {
                const float dt = P.tgt.depth[gp];
                if (dt > 0.f) g = a_d * sgn(P.depth[gp] - dt);
            }
            P.g.depth[gp] = g;
        }
        if (P.g.kmap) P.g.kmap[gp] = P.kmap ? a_k * sgn(P.kmap[gp] - 1.f) : 0.f;
        if (NS > 0 && P.g.logits) {
            constexpr int N1 = NS > 0 ? NS : 1;
            float* G = P.g.logits + po * P.n_sem + idx;
            const int lab = P.tgt.label ? P.tgt.label[gp] : -1;
            if (lab >= 0 && lab < P.n_sem) {
                float o[N1], mx, z;
                pixel_logits<N1>(P.logits + po * P.n_sem + idx, hw, P.n_sem, o, &mx, &z);
                const float iz = a_s / z;
#pragma unroll
                for (int c = 0; c < N1; ++c)
                    if (c < P.n_sem) {
                        const float p = expf(o[c] - mx) * iz;
                        G[(int64_t)c * hw] = c == lab ? p - a_s : p;
                    }
            } else {
#pragma unroll
                for (int c = 0; c < N1; ++c)
                    if (c < P.n_sem) G[(int64_t)c * hw] = 0.f;
            }
        }
    }
}

template <int NS>
static void launch_loss_t(const LossParams& P, int blocks, cudaStream_t st) {
    loss_sums_kernel<NS><<<(unsigned)blocks, LOSS_THREADS, 0, st>>>(P);
    loss_finalize_kernel<<<1, LOSS_THREADS, 0, st>>>(P, blocks);
    loss_grad_kernel<NS><<<(unsigned)blocks, LOSS_THREADS, 0, st>>>(P);
}

int launch_loss(const unigs_plan& p, const unigs_outputs& out, const float* normal_d,
                const unigs_targets& tgt, const unigs_loss_lambda& lam, void* ws, float* record,
                const unigs_loss_grads& g, cudaStream_t st) {
    LossParams P;
    P.n_cams = p.n_cams;
    P.n_sem = p.n_sem;
    P.n_pixels = p.n_pixels;
    for (int k = 0; k <= UNIGS_MAX_CAMS; ++k) P.pix_off[k] = k <= p.n_cams ? p.pixel_offset[k] : 0;
    P.rgb = out.rgb;
    P.depth = out.depth;
    P.kmap = out.kmap;
    P.logits = out.logits;
    P.normal_d = normal_d;
    P.tgt = tgt;
    P.lam = lam;
    P.partial = ws_ptr<float>(ws, p, OFF_LOSS);
    P.record = record;
    P.g = g;
    int64_t blocks = (p.n_pixels + LOSS_THREADS - 1) / LOSS_THREADS;
    const int64_t cap = (int64_t)sm_count() * 4;
    if (blocks > cap) blocks = cap;
    if (blocks > LOSS_MAX_BLOCKS) blocks = LOSS_MAX_BLOCKS;
    if (blocks < 1) blocks = 1;
    // logits of a pixel are held in registers: the kernels are compiled for
    // 8, 16, 32 and 64 channels
    if (p.n_sem == 0)
        launch_loss_t<0>(P, (int)blocks, st);
    else if (p.n_sem <= 8)
        launch_loss_t<8>(P, (int)blocks, st);
    else if (p.n_sem <= 16)
        launch_loss_t<16>(P, (int)blocks, st);
    else if (p.n_sem <= 32)
        launch_loss_t<32>(P, (int)blocks, st);
    else
        launch_loss_t<64>(P, (int)blocks, st);
    return 3;
}

// -------------------------------------------------------------------- Adam
struct AdamParams {
    unigs_adam_group grp[UNIGS_ADAM_MAX_GROUPS];
    int n_groups;
    float beta1, beta2, eps;
    const int32_t* step;
};

// One element of the update (or, without UPDATE, of the copies only).
template <bool UPDATE>
__device__ __forceinline__ float adam_one(float raw, float g, float& m, float& v, int act,
                                          float lr, float b1, float b2, float eps, float bc1,
                                          float bc2) {
    if (UPDATE) {
        if (act == UNIGS_ACT_EXP) {
            g *= expf(raw);
        } else if (act == UNIGS_ACT_SIGMOID) {
            const float s = 1.f / (1.f + expf(-raw));
            g *= s * (1.f - s);
        }
        m = b1 * m + (1.f - b1) * g;
        v = b2 * v + (1.f - b2) * g * g;
        raw -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    }
    return raw;
}

__device__ __forceinline__ float activate(float raw, int act) {
    if (act == UNIGS_ACT_EXP) return expf(raw);
    if (act == UNIGS_ACT_SIGMOID) return 1.f / (1.f + expf(-raw));
    return raw;
}

template <bool UPDATE>
__global__ void __launch_bounds__(256) adam_kernel(const __grid_constant__ AdamParams P) {
    const unigs_adam_group& G = P.grp[blockIdx.y];
    const int t = UPDATE ? P.step[0] + 1 : 1;
    const float bc1 = 1.f - powf(P.beta1, (float)t);
    const float bc2 = 1.f - powf(P.beta2, (float)t);
    const float lr = G.lr;
    const int act = G.activation;
    const float b1 = P.beta1, b2 = P.beta2, eps = P.eps;
    // 16-byte vectors where every array allows it (bfloat16 copies: 8 bytes)
    const uintptr_t al = reinterpret_cast<uintptr_t>(G.param) |
                         (UPDATE ? reinterpret_cast<uintptr_t>(G.grad) |
                                       reinterpret_cast<uintptr_t>(G.m) |
                                       reinterpret_cast<uintptr_t>(G.v)
                                 : 0) |
                         reinterpret_cast<uintptr_t>(G.act_out);
    const bool vec = (al & 15) == 0 && (reinterpret_cast<uintptr_t>(G.bf16_out) & 7) == 0;
    const int64_t n4 = vec ? G.count / 4 : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 raw = reinterpret_cast<const float4*>(G.param)[i];
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f), m = g, v = g;
        if (UPDATE) {
            g = reinterpret_cast<const float4*>(G.grad)[i];
            m = reinterpret_cast<const float4*>(G.m)[i];
            v = reinterpret_cast<const float4*>(G.v)[i];
        }
        raw.x = adam_one<UPDATE>(raw.x, g.x, m.x, v.x, act, lr, b1, b2, eps, bc1, bc2);
        raw.y = adam_one<UPDATE>(raw.y, g.y, m.y, v.y, act, lr, b1, b2, eps, bc1, bc2);
        raw.z = adam_one<UPDATE>(raw.z, g.z, m.z, v.z, act, lr, b1, b2, eps, bc1, bc2);
        raw.w = adam_one<UPDATE>(raw.w, g.w, m.w, v.w, act, lr, b1, b2, eps, bc1, bc2);
        if (UPDATE) {
            reinterpret_cast<float4*>(G.param)[i] = raw;
            reinterpret_cast<float4*>(G.m)[i] = m;
            reinterpret_cast<float4*>(G.v)[i] = v;
        }
        const float4 a = make_float4(activate(raw.x, act), activate(raw.y, act),
                                     activate(raw.z, act), activate(raw.w, act));
        if (G.act_out) reinterpret_cast<float4*>(G.act_out)[i] = a;
        if (G.bf16_out) {
            const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a.x)) |
                                ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a.y)) << 16);
            const uint32_t hi = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a.z)) |
                                ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a.w)) << 16);
            reinterpret_cast<uint2*>(G.bf16_out)[i] = make_uint2(lo, hi);
        }
    }
    // scalar elements (the tail, or everything without vector alignment)
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.count;
         i += stride) {
        float m = 0.f, v = 0.f, g = 0.f;
        if (UPDATE) {
            g = G.grad[i];
            m = G.m[i];
            v = G.v[i];
        }
        const float raw = adam_one<UPDATE>(G.param[i], g, m, v, act, lr, b1, b2, eps, bc1, bc2);
        if (UPDATE) {
            G.param[i] = raw;
            G.m[i] = m;
            G.v[i] = v;
        }
        const float a = activate(raw, act);
        if (G.act_out) G.act_out[i] = a;
        if (G.bf16_out) reinterpret_cast<__nv_bfloat16*>(G.bf16_out)[i] = __float2bfloat16_rn(a);
    }
}

__global__ void adam_step_store_kernel(int32_t* step) { step[0] += 1; }

static AdamParams adam_params(const unigs_adam_group* groups, int n_groups,
                              const unigs_adam_hparams* hp, const int32_t* step, int64_t* most) {
    AdamParams P;
    *most = 0;
    for (int i = 0; i < n_groups; ++i) {
        P.grp[i] = groups[i];
        if (groups[i].count > *most) *most = groups[i].count;
    }
    P.n_groups = n_groups;
    P.beta1 = hp ? hp->beta1 : 0.f;
    P.beta2 = hp ? hp->beta2 : 0.f;
    P.eps = hp ? hp->eps : 0.f;
    P.step = step;
    return P;
}

static unsigned adam_blocks(int64_t most) {
    int64_t bx = (most / 4 + 255) / 256 + 1;
    const int64_t cap = (int64_t)sm_count() * 8;
    return (unsigned)(bx > cap ? cap : bx);
}

int launch_adam(const unigs_adam_group* groups, int n_groups, const unigs_adam_hparams& hp,
                int32_t* step, cudaStream_t st) {
    int64_t most;
    const AdamParams P = adam_params(groups, n_groups, &hp, step, &most);
    int launches = 0;
    if (n_groups > 0 && most > 0) {
        adam_kernel<true><<<dim3(adam_blocks(most), (unsigned)n_groups), 256, 0, st>>>(P);
        ++launches;
    }
    adam_step_store_kernel<<<1, 1, 0, st>>>(step);
    return launches + 1;
}

int launch_param_copies(const unigs_adam_group* groups, int n_groups, cudaStream_t st) {
    int64_t most;
    const AdamParams P = adam_params(groups, n_groups, nullptr, nullptr, &most);
    if (n_groups == 0 || most == 0) return 0;
    adam_kernel<false><<<dim3(adam_blocks(most), (unsigned)n_groups), 256, 0, st>>>(P);
    return 1;
}

// ----------------------------------------------------------------- pruning
struct PruneWs {
    uint32_t* keep;
    uint32_t* pos;
    uint32_t* partial;
    uint32_t* count;
};

inline PruneWs prune_ws_layout(void* ws, int64_t n) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* b = static_cast<char*>(ws);
    PruneWs w;
    size_t o = 0;
    w.count = reinterpret_cast<uint32_t*>(b + o);
    o += 256;
    w.keep = reinterpret_cast<uint32_t*>(b + o);
    o += up(sizeof(uint32_t) * (size_t)n);
    w.pos = reinterpret_cast<uint32_t*>(b + o);
    o += up(sizeof(uint32_t) * (size_t)n);
    w.partial = reinterpret_cast<uint32_t*>(b + o);
    return w;
}

size_t prune_ws_bytes(int64_t n) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nb = (size_t)((n + SCAN_ITEMS - 1) / SCAN_ITEMS) + 1;
    return 256 + 2 * up(sizeof(uint32_t) * (size_t)n) + up(sizeof(uint32_t) * nb);
}

__global__ void __launch_bounds__(256) prune_mark_kernel(const float* __restrict__ k, int64_t n,
                                                         float T_k, uint32_t* __restrict__ keep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keep[i] = fabsf(k[i] - 1.f) > T_k ? 0u : 1u;
}

template <typename E>
__global__ void __launch_bounds__(256)
    prune_compact_kernel(const E* __restrict__ src, E* __restrict__ dst, int64_t n, int64_t n_keep,
                         int planes, int row, const uint32_t* __restrict__ keep,
                         const uint32_t* __restrict__ pos, int fill, float fill_value) {
    const int64_t per_plane = n * (int64_t)row;
    const int64_t total = per_plane * planes;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pl = e / per_plane;
        const int64_t r = e - pl * per_plane;
        const int64_t i = r / row;
        const int64_t c = r - i * row;
        if (!keep[i]) continue;
        const int64_t d = (pl * n_keep + pos[i]) * row + c;
        if (fill)
            reinterpret_cast<float*>(dst)[d] = fill_value;
        else
            dst[d] = src[e];
    }
}

int launch_prune_mark(const float* k, int64_t n, float T_k, void* ws, cudaStream_t st) {
    PruneWs w = prune_ws_layout(ws, n);
    cudaMemsetAsync(w.count, 0, sizeof(uint32_t), st);
    if (n == 0) return 0;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    prune_mark_kernel<<<(unsigned)blocks, 256, 0, st>>>(k, n, T_k, w.keep);
    return 1 + scan_u32(w.keep, n, w.partial, w.pos, w.count, st);
}

uint32_t* prune_count_ptr(void* ws, int64_t n) { return prune_ws_layout(ws, n).count; }

int launch_prune_compact(const unigs_prune_array* arrays, int n_arrays, int64_t n, int64_t n_keep,
                         const void* ws, cudaStream_t st) {
    PruneWs w = prune_ws_layout(const_cast<void*>(ws), n);
    int launches = 0;
    for (int a = 0; a < n_arrays; ++a) {
        const unigs_prune_array& A = arrays[a];
        const int64_t total = n * (int64_t)A.row * A.planes;
        if (total == 0 || n_keep == 0) continue;
        int64_t blocks = (total + 255) / 256;
        const int64_t cap = (int64_t)sm_count() * 8;
        if (blocks > cap) blocks = cap;
        if (A.elem_bytes == 4)
            prune_compact_kernel<uint32_t><<<(unsigned)blocks, 256, 0, st>>>(
                static_cast<const uint32_t*>(A.src), static_cast<uint32_t*>(A.dst), n, n_keep,
                A.planes, A.row, w.keep, w.pos, A.fill, A.fill_value);
        else
            prune_compact_kernel<uint16_t><<<(unsigned)blocks, 256, 0, st>>>(
                static_cast<const uint16_t*>(A.src), static_cast<uint16_t*>(A.dst), n, n_keep,
                A.planes, A.row, w.keep, w.pos, 0, 0.f);
        ++launches;
    }
    return launches;
}

}  // namespace unigs
