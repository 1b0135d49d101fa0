// Backward composite (Alg. 4) with the semantic terms on the 5th-generation
// tensor cores, for bfloat16 logit storage.
//
// The per-pair work of the reverse walk (T restoration, dL/dalpha, the splat
// and ray-ellipsoid chain, the 32-entry gradient record) is that of the
// FP32-pipe kernel (render_bwd.cu, bwd_pair.cuh).  What moves to the tensor
// core are the two products of the semantic channel, per tile and batch of
// B = 16 Gaussians:
//   MMA 1 (before the walk of the batch): the logit part of G_i,
//     Gsem[p][j] = sum_c gO[p][c] F[j][c]              (Eq. gradiento, Alg. 4)
//     M = 128 pixels (two M-tiles), N = B, K = the tile's upstream rows;
//   MMA 2 (after the walk): the logit-feature gradient
//     dL/dF[j][c] = sum_p w[p][j] gO[p][c]              (Eq. gradiento)
//     M = 128 channel rows, N = B, K = 256 pixels;
// one atomic per (Gaussian, channel, tile and split) then replaces the
// FP32-pipe kernel's per-warp channel gather.
//
// Precision: both products run on float16 operands split into hi + lo parts
// (x = hi + lo + r, |r| <= 2^-22 |x| in float16's normal range), with exact
// power-of-two scales that put every operand there: the upstream tile is
// scaled by 2^kg (its largest |gO| to [2^13, 2^14)), each batch's F by 2^kf
// (F's bfloat16 values then convert to float16 exactly), and w by 2^14.  The
// upstream logit gradient is stored once per tile as 128 K-entries per pixel:
// NS hi, NS lo, zero padding.  MMA 1 runs K over both halves against the same
// F chunks, so Gsem = (hi + lo) . F; MMA 2 takes the 128 entries as its M rows
// (hi rows then lo rows) and W = w_hi + w_lo as two K passes, and the two row
// halves of a channel are added by the atomics.  Products are exact and
// accumulate in float32 in tensor memory; the scales are undone (exactly) on
// read-back.  Each product term thus carries at most ~2^-21 relative error,
// below the float32 rounding of the FP32-pipe kernel's own dot products.
//
// Layout (bytes; K-major operands are 8-row x 16-byte core matrices, lbo the
// stride between core matrices along K, sbo along M or N):
//   ga: upstream tile, pixel p's 16 chunks (8 K-entries each) at
//       (p / 8) * 2048 + chunk * 128 + (p % 8) * 16: K-major for MMA 1
//       (M = pixels: lbo 128, sbo 2048) and, read transposed, MN-major for
//       MMA 2 (M = K-entries along a row: sbo 128; K = pixels: lbo 2048);
//   wb: W^T per split, K-major (N = Gaussians, K = pixels): Gaussian j,
//       pixel p at (j / 8) * 4096 + (p / 8) * 128 + (j % 8) * 16 + (p % 8) * 2;
//   fb: F, K-major (N = Gaussians, K = channels), re-laid from the staged
//       rows by the staging warp.
// Tensor memory (float32 accumulators): Gsem for (buffer, M-tile) at column (2 buffer + M-tile) B,
// dL/dF for buffer at column 4 B + buffer B; pixel thread tid owns lane tid %
// 128 of M-tile tid / 128.
//
// Warps 0-7 walk the pixels (one pixel per thread, as in the FP32-pipe
// kernel); warp 8 stages each batch (bulk copies of the records and logit
// rows), re-lays F, and issues both MMAs.  Per batch and operand buffer the
// handshake is: staged (bar) -> MMA 1 done (d1_bar) -> every pixel warp
// walked the batch and wrote its W entries (wrdy, 8 arrivals) -> MMA 2 done
// (d2_bar).  Buffers alternate, so the staging warp prepares batch i + 1
// while the pixel warps walk batch i, and a pixel warp reads back the
// feature gradients of batch i - 2 (whose W buffer it is about to rewrite).
#include <cuda_fp16.h>

#include "bwd_pair.cuh"
#include "launch.h"
#include "tcgen05.cuh"

namespace unigs {

constexpr uint32_t BTC_WAIT_LIMIT = 1u << 22;
constexpr int BTC_BATCH = 16;
constexpr int BTC_THREADS = 288;
constexpr int BTC_CTAS_PER_SM = 2;

struct BwdTcParams {
    const CamTable* tab;
    int n_cams;
    int n_sem;
    int64_t n;
    int64_t n_tiles;
    const float* rec;
    const __nv_bfloat16* sem;  // rows [n][n_sem]
    const uint32_t* vals;
    const uint2* ranges;
    const uint32_t* order;
    uint32_t* work;
    WsHeader* hdr;
    const float* T_final;
    const uint32_t* n_contrib;
    unigs_grad_outputs go;
    double* grec;
    float* gsem;
    float alpha_min, alpha_max;
    int center_depth;
    int sem_bulk;
};

template <int NS>
struct BwdTcSmem {
    static constexpr int B = BTC_BATCH;
    static constexpr int KCH = 16;               // 16-byte K chunks per pixel row of ga
    static constexpr int SBO_G = KCH * 128;      // between 8-pixel groups of ga
    static constexpr int SBO_W = 32 * 128;       // between 8-Gaussian groups of W^T
    static constexpr int W_BYTES = B * 256 * 2;  // one split of W^T
    static constexpr int SBO_F = (NS / 8) * 128; // between 8-Gaussian groups of F
    static_assert(2 * NS <= 8 * KCH, "the upstream rows hold NS hi and NS lo entries");
    __align__(1024) unsigned char ga[32 * SBO_G];
    __align__(128) unsigned char wb[2][2][W_BYTES];  // [buffer][split]
    __align__(128) unsigned char fb[2][(B / 8) * SBO_F];
    __align__(16) float rec[2][B][REC_FLOATS];
    __align__(16) __nv_bfloat16 semraw[2][B][NS];  // staged logit rows
    uint32_t ids[4][B];  // Gaussian ids per batch (ring of 4: read back two batches later)
    uint64_t bar[2];     // batch staged (bulk bytes + the staging warp's arrival)
    uint64_t d1_bar[2];  // MMA 1 of the buffer complete
    uint64_t wrdy[2];    // the 8 pixel warps are done with the batch (8 arrivals)
    uint64_t d2_bar[2];  // MMA 2 of the buffer complete
    float finv[2];       // 2^-kf of the buffer's batch (released by the staging warp's
                         // own arrival on d1_bar)
    uint32_t tmem_base;
    uint32_t max_last;
    uint32_t gmax;       // bits of the tile's largest |gO| (non-negative floats order as uints)
    int tile;
    uint32_t issued[2];  // staging phases started per buffer
};

// Exponent k such that m 2^k lies in [2^13, 2^14) for m > 0 (clamped to
// +-125, so that 2^k and 2^-k are normal floats); 0 for m = 0.
__device__ __forceinline__ int scale_exp(float m) {
    if (!(m > 0.f)) return 0;
    const int e = (int)((__float_as_uint(m) >> 23) & 255u) - 126;  // m = f 2^e, f in [0.5, 1)
    return max(-125, min(125, 14 - e));
}
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

// x = hi + lo as two float16 (packed pairs for two values).
__device__ __forceinline__ void split_f16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
    hi = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
    lo = (uint32_t)__half_as_ushort(__float2half_rn(x0 - __half2float(h0))) |
         ((uint32_t)__half_as_ushort(__float2half_rn(x1 - __half2float(h1))) << 16);
}

// Bounded wait that is skipped once this thread has given up.
__device__ __forceinline__ void btc_wait(uint64_t* bar, uint32_t parity, bool& timed_out) {
    if (!timed_out && !mbar_wait_bounded(bar, parity, BTC_WAIT_LIMIT)) timed_out = true;
}

template <int NS>
__device__ __forceinline__ void btc_stage(const BwdTcParams& P, BwdTcSmem<NS>& S, int buf,
                                          int slot, uint32_t first, int count, int cam) {
    // executed by the staging warp
    const int lane = threadIdx.x & 31;
    const uint32_t row_bytes = (uint32_t)(P.n_sem * 2);
    const uint32_t per = REC_FLOATS * 4 + (P.sem_bulk ? row_bytes : 0u);
    if (lane == 0) mbar_expect_tx(&S.bar[buf], per * (uint32_t)count);
    __syncwarp();
    for (int i = lane; i < count; i += 32) {
        const uint32_t g = P.vals[first + i];
        S.ids[slot][i] = g;
        const size_t r = (size_t)cam * (size_t)P.n + g;
        bulk_g2s(&S.rec[buf][i][0], P.rec + r * REC_FLOATS, REC_FLOATS * 4, &S.bar[buf]);
        const __nv_bfloat16* src = P.sem + (size_t)g * P.n_sem;
        if (P.sem_bulk)
            bulk_g2s(&S.semraw[buf][i][0], src, row_bytes, &S.bar[buf]);
        else
            for (int c = 0; c < P.n_sem; ++c) S.semraw[buf][i][c] = src[c];
    }
    // the plain stores (ids, unaligned rows) are released by this arrival
    __syncwarp();
    if (lane == 0) {
        mbar_arrive(&S.bar[buf]);
        ++S.issued[buf];
    }
}

template <int NS>
__global__ void __launch_bounds__(BTC_THREADS, BTC_CTAS_PER_SM)
    render_bwd_tc_kernel(const BwdTcParams P) {
    using Sm = BwdTcSmem<NS>;
    constexpr int B = BTC_BATCH;
    constexpr uint32_t NCOLS = 128;  // Gsem 4 B + dL/dF 2 B = 96 columns
    constexpr uint32_t IDESC1 = idesc_f16_f32(128, B);
    constexpr uint32_t IDESC2 = idesc_f16_f32(128, B) | IDESC_A_MN;
    constexpr float W_SCALE = 16384.f, W_UNSCALE = 1.f / 16384.f;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Sm& S = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool stager = warp == 8;

    // once per CTA: zero the logit staging (rows shorter than NS stay zero),
    // init barriers, allocate the tensor-memory columns
    for (int j = tid; j < 2 * B * NS; j += BTC_THREADS)
        (&S.semraw[0][0][0])[j] = __float2bfloat16_rn(0.f);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.bar[b], 1);
            mbar_init(&S.d1_bar[b], 2);  // the MMA commit + the staging warp
            mbar_init(&S.wrdy[b], 8);
            mbar_init(&S.d2_bar[b], 1);
        }
        fence_mbar_init();
        S.issued[0] = S.issued[1] = 0u;
    }
    if (warp == 0) {
        tmem_alloc(&S.tmem_base, NCOLS);
        tmem_relinquish();
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = S.tmem_base;
    // this pixel thread's tensor-memory lane and M-tile
    const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
    const int mt = (warp >> 2) & 1;

    bool timed_out = false;
    uint32_t gb = 0;                  // batches begun by this CTA (uniform)
    // MMA commits per buffer (staging warp), scalars so they stay in registers
    uint32_t c1a = 0u, c1b = 0u, c2a = 0u, c2b = 0u;

    for (;;) {
        if (tid == 0) {
            S.tile = (int)atomicAdd(P.work, 1u);
            S.max_last = 0;
            S.gmax = 0;
        }
        __syncthreads();
        const int64_t t = S.tile;
        if (t >= P.n_tiles) break;
        const int64_t gtile = P.order[t];
        int cam_idx;
        const DevCam& cam = cam_of_tile(P.tab, P.n_cams, gtile, &cam_idx);
        const int64_t ltile = gtile - cam.tile_off;
        const int tx = (int)(ltile % cam.tiles_x), ty = (int)(ltile / cam.tiles_x);
        const int tw = cam.tile_w, th = cam.tile_h;
        const uint2 range = P.ranges[gtile];

        // pixel state (warps 0-7)
        int lx = 0, ly = 0, wbx = 0, wby = 0;
        const int ptid = tid & 255;
        tile_pixel(ptid, tw, &lx, &ly);
        warp_block(warp & 7, tw, &wbx, &wby);
        const int u = tx * tw + lx, v = ty * th + ly;
        const float bx0 = (float)(tx * tw + wbx);
        const float by0 = (float)(ty * th + wby);
        const bool inside = !stager && u < cam.width && v < cam.height;
        const float uf = (float)u, vf = (float)v;
        const float xt = (uf - cam.cx) / cam.fx, yt = (vf - cam.cy) / cam.fy;
        const int W = cam.width;
        const int64_t HW = (int64_t)cam.height * W;
        const int64_t pix = cam.pix_off;
        const int64_t idx = (int64_t)v * W + u;
        float T = 1.f;
        uint32_t last = 0;
        PixelUp up = {{0.f, 0.f, 0.f}, 0.f, {0.f, 0.f, 0.f}, 0.f};
        const float* g_log = P.go.logits ? P.go.logits + pix * (int64_t)P.n_sem + idx : nullptr;
        if (!stager) {
            // the tile's largest upstream logit gradient (for its scale)
            float gm = 0.f;
            if (inside && g_log)
                for (int c = 0; c < P.n_sem; ++c) gm = fmaxf(gm, fabsf(g_log[c * HW]));
            if (gm > 0.f) atomicMax(&S.gmax, __float_as_uint(gm));
            if (inside) {
                T = P.T_final[pix + idx];
                last = P.n_contrib[pix + idx];
                load_pixel_up(P.go, pix, HW, idx, up);
            }
            if (last) atomicMax(&S.max_last, last);
        }
        const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);
        __syncthreads();
        const int kg = scale_exp(__uint_as_float(S.gmax));
        const float ginv = pow2f(-kg);
        if (!stager) {
            // the pixel's upstream logit gradients x 2^kg as float16 hi / lo
            // K-entries
            const float sg = pow2f(kg);
            unsigned char* grow = S.ga + (ptid >> 3) * Sm::SBO_G + (ptid & 7) * 16;
#pragma unroll
            for (int kc = 0; kc < NS / 8; ++kc) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float f[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int c = 8 * kc + 2 * e + q;
                        f[q] = (inside && g_log && c < P.n_sem) ? g_log[c * HW] * sg : 0.f;
                    }
                    split_f16x2(f[0], f[1], h[e], l[e]);
                }
                *reinterpret_cast<uint4*>(grow + kc * 128) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(grow + (NS / 8 + kc) * 128) =
                    make_uint4(l[0], l[1], l[2], l[3]);
            }
#pragma unroll
            for (int kc = NS / 4; kc < Sm::KCH; ++kc)
                *reinterpret_cast<uint4*>(grow + kc * 128) = make_uint4(0u, 0u, 0u, 0u);
            fence_async_shared();
        }
        __syncthreads();
        const int n_items = (int)S.max_last;
        const int n_batches = (n_items + B - 1) / B;
        const uint32_t gb0 = gb;
        gb += (uint32_t)n_batches;

        if (stager) {
            // ------------------------------------------------ staging warp
            auto mma2 = [&](uint32_t gk) {
                const int bf = (int)(gk & 1u);
                btc_wait(&S.wrdy[bf], (gk >> 1) & 1u, timed_out);
                if (__any_sync(0xffffffffu, timed_out)) {
                    timed_out = true;
                    return;
                }
                if (lane == 0) {
                    tc_fence_after_sync();
                    const uint32_t d = tmem + 4 * B + (uint32_t)(bf * B);
#pragma unroll 1
                    for (int ks = 0; ks < 16; ++ks) {
                        const uint64_t a = smem_desc_kmajor(S.ga + ks * 2 * Sm::SBO_G,
                                                            Sm::SBO_G, 128);
#pragma unroll
                        for (int s = 0; s < 2; ++s) {
                            const uint64_t w = smem_desc_kmajor(&S.wb[bf][s][0] + ks * 256, 128,
                                                                Sm::SBO_W);
                            mma_bf16(d, a, w, IDESC2, (ks > 0 || s > 0) ? 1u : 0u);
                        }
                    }
                    mma_commit(&S.d2_bar[bf]);
                }
                if (bf) ++c2b; else ++c2a;
            };
            for (int it = 0; it < n_batches; ++it) {
                const int b = n_batches - 1 - it;
                const uint32_t gk = gb0 + (uint32_t)it;
                const int bf = (int)(gk & 1u);
                // the buffer's previous batch is done (its MMA 2 was issued
                // after the same wait)
                if (gk >= 2) btc_wait(&S.wrdy[bf], ((gk >> 1) - 1) & 1u, timed_out);
                if (__any_sync(0xffffffffu, timed_out)) {
                    timed_out = true;
                    break;
                }
                const int count = min(B, n_items - b * B);
                btc_stage<NS>(P, S, bf, (int)(gk & 3u), range.x + (uint32_t)(b * B), count,
                              cam_idx);
                btc_wait(&S.bar[bf], (gk >> 1) & 1u, timed_out);
                if (__any_sync(0xffffffffu, timed_out)) {
                    timed_out = true;
                    break;
                }
                // F x 2^kf as float16 (exact) in K-major core matrices: row j,
                // channels 8 kc .. 8 kc + 7; kf from the batch's largest |f|
                uint32_t fm = 0u;
                for (int task = lane; task < count * (NS / 8); task += 32) {
                    const int j = task / (NS / 8), kc = task % (NS / 8);
                    const __nv_bfloat16* src = &S.semraw[bf][j][8 * kc];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        fm = max(fm, __float_as_uint(fabsf(__bfloat162float(src[e]))));
                }
                fm = __reduce_max_sync(0xffffffffu, fm);
                const int kf = scale_exp(__uint_as_float(fm));
                const float sf = pow2f(kf);
                for (int task = lane; task < B * (NS / 8); task += 32) {
                    const int j = task / (NS / 8), kc = task % (NS / 8);
                    const __nv_bfloat16* src = &S.semraw[bf][j][8 * kc];
                    uint32_t q[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        q[e] = (uint32_t)__half_as_ushort(
                                   __float2half_rn(__bfloat162float(src[2 * e]) * sf)) |
                               ((uint32_t)__half_as_ushort(
                                    __float2half_rn(__bfloat162float(src[2 * e + 1]) * sf)) << 16);
                    *reinterpret_cast<uint4*>(&S.fb[bf][0] + (j >> 3) * Sm::SBO_F + kc * 128 +
                                              (j & 7) * 16) = make_uint4(q[0], q[1], q[2], q[3]);
                }
                if (lane == 0) S.finv[bf] = pow2f(-kf);
                fence_async_shared();
                __syncwarp();
                if (lane == 0) {
                    tc_fence_after_sync();
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const uint32_t d = tmem + (uint32_t)((2 * bf + m) * B);
#pragma unroll
                        for (int ks = 0; ks < NS / 8; ++ks) {
                            // K-entries 16 ks .. 16 ks + 15: hi channels for the
                            // first NS / 16 steps, then lo, both against F
                            const uint64_t a = smem_desc_kmajor(
                                S.ga + m * 16 * Sm::SBO_G + ks * 256, 128, Sm::SBO_G);
                            const uint64_t f = smem_desc_kmajor(
                                &S.fb[bf][0] + (ks % (NS / 16)) * 256, 128, Sm::SBO_F);
                            mma_bf16(d, a, f, IDESC1, ks > 0 ? 1u : 0u);
                        }
                    }
                    mma_commit(&S.d1_bar[bf]);
                    mbar_arrive(&S.d1_bar[bf]);  // releases S.finv[bf]
                }
                if (bf) ++c1b; else ++c1a;
                if (it > 0) mma2(gk - 1u);
                if (timed_out) break;
            }
            if (n_batches > 0 && !timed_out) mma2(gb0 + (uint32_t)n_batches - 1u);
        } else {
            // ------------------------------------------------ pixel warps
            float Sacc = 0.f;
            // this thread's W^T entries: Gaussian j at wcol + (j / 8) SBO_W + (j % 8) 16
            const int wcol = (ptid >> 3) * 128 + (ptid & 7) * 2;
            // channel row of this lane in the dL/dF read-back, and its first column
            const int crow = 32 * (warp & 3) + lane;
            const int cch = crow < NS ? crow : crow - NS;
            const bool crow_ok = crow < 2 * NS && cch < P.n_sem;
            const int ccol = (warp >> 2) * 8;
            // adds the feature gradients of batch gk (MMA 2 complete) to dL/dF
            auto readback = [&](uint32_t gk, int count) {
                const int bf = (int)(gk & 1u);
                btc_wait(&S.d2_bar[bf], (gk >> 1) & 1u, timed_out);
                if (__any_sync(0xffffffffu, timed_out)) {
                    timed_out = true;
                    return;
                }
                tc_fence_after_sync();
                float dv[8];
                tmem_ld8(tmem + lane_addr + 4 * B + (uint32_t)(bf * B + ccol), dv);
                if (crow_ok) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = ccol + q;
                        if (j < count && dv[q] != 0.f)
                            atomicAdd(P.gsem + (size_t)S.ids[gk & 3u][j] * P.n_sem + cch,
                                      dv[q] * ginv * W_UNSCALE);
                    }
                }
            };
            for (int it = 0; it < n_batches; ++it) {
                const int b = n_batches - 1 - it;
                const uint32_t gk = gb0 + (uint32_t)it;
                const int bf = (int)(gk & 1u);
                btc_wait(&S.bar[bf], (gk >> 1) & 1u, timed_out);
                btc_wait(&S.d1_bar[bf], (gk >> 1) & 1u, timed_out);
                if (__any_sync(0xffffffffu, timed_out)) timed_out = true;
                tc_fence_after_sync();
                // the W^T buffer of this batch was last read by MMA 2 of batch
                // it - 2: add that batch's feature gradients, then rewrite it
                if (it >= 2) readback(gk - 2u, min(B, n_items - (b + 2) * B));
                unsigned char* w0 = &S.wb[bf][0][0];
                unsigned char* w1 = &S.wb[bf][1][0];
                {
                    // zero the warp's W^T entries: pixel groups 4 w .. 4 w + 3,
                    // for both splits, every Gaussian row
                    const int pw = warp & 7;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = lane + 32 * q;  // 128 chunks of 16 bytes
                        const int s = i >> 6, jg = (i >> 5) & 1, r = (i >> 2) & 7,
                                  pg = 4 * pw + (i & 3);
                        *reinterpret_cast<uint4*>(&S.wb[bf][s][0] + jg * Sm::SBO_W + pg * 128 +
                                                  r * 16) = make_uint4(0u, 0u, 0u, 0u);
                    }
                    __syncwarp();
                }
                const int count = min(B, n_items - b * B);
                const uint32_t d1 = tmem + lane_addr + (uint32_t)((2 * bf + mt) * B);
                const float finv = S.finv[bf];
                if (!__all_sync(0xffffffffu, timed_out) && (uint32_t)(b * B) < wlast) {
                    for (int j = min(count, (int)(wlast - (uint32_t)(b * B))) - 1; j >= 0; --j) {
                        const uint32_t pos = (uint32_t)(b * B + j);
                        const float* rc = &S.rec[bf][j][0];
                        if (warp_block_misses(rc, bx0, by0)) continue;  // uniform per warp
                        // Gsem of this pixel and Gaussian, loaded while alpha is evaluated
                        const uint32_t gsem_raw = tmem_ld1_issue(d1 + (uint32_t)j);
                        float dx, dy, Gs, wq;
                        const float alpha = splat_alpha(rc, uf, vf, P.alpha_max, &dx, &dy, &Gs, &wq);
                        const float gsem = tmem_ld1_wait(gsem_raw);
                        const bool contrib = !timed_out && pos < last && alpha >= P.alpha_min;
                        if (!__any_sync(0xffffffffu, contrib)) continue;
                        const float G_sem = gsem * ginv * finv;
                        float gv[32];
                        const float w = bwd_pair(rc, up, xt, yt, wq, dx, dy, alpha, Gs,
                                                 contrib, G_sem, P.alpha_max, P.center_depth, T,
                                                 Sacc, gv);
                        if (contrib) {
                            // w 2^14 = hi + lo, both float16, in W^T column j
                            const float ws = w * W_SCALE;
                            const __half wh = __float2half_rn(ws);
                            const int off = wcol + (j >> 3) * Sm::SBO_W + (j & 7) * 16;
                            *reinterpret_cast<__half*>(w0 + off) = wh;
                            *reinterpret_cast<__half*>(w1 + off) =
                                __float2half_rn(ws - __half2float(wh));
                        }
                        const uint32_t g = S.ids[gk & 3u][j];
                        const size_t rix = (size_t)cam_idx * (size_t)P.n + g;
                        // the warp's sum of component `lane`, added in float64
                        // (see the FP32-pipe kernel)
                        const float tot = warp_reduce_transpose32(gv, lane);
                        if (tot != 0.f) atomicAdd(P.grec + rix * GREC_FLOATS + lane, (double)tot);
                    }
                }
                // this warp is done with the batch's records, Gsem and W^T
                fence_async_shared();
                tc_fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.wrdy[bf]);
            }
            // the last two batches' feature gradients
            for (int it = max(0, n_batches - 2); it < n_batches; ++it) {
                const int b = n_batches - 1 - it;
                readback(gb0 + (uint32_t)it, min(B, n_items - b * B));
            }
            tc_fence_before_sync();
        }
        // a bounded wait that gave up ends the CTA (uniformly)
        if (__syncthreads_or(timed_out)) break;
        tc_fence_after_sync();
    }
    // Before the CTA exits: no bulk copy may still be landing in its shared
    // memory and no MMA may still be running on its operands or columns (the
    // staging warp waits, bounded, for the last staging phase and the last
    // commit of each barrier); then the columns are returned.
    if (stager) {
        if (lane == 0 && !drain_bulk(S.bar, S.issued[0], S.issued[1], BTC_WAIT_LIMIT))
            timed_out = true;
        const uint32_t c1[2] = {c1a, c1b}, c2[2] = {c2a, c2b};
#pragma unroll
        for (int bf = 0; bf < 2; ++bf) {
            if (c1[bf] > 0 && !mbar_wait_bounded(&S.d1_bar[bf], (c1[bf] - 1) & 1u, BTC_WAIT_LIMIT))
                timed_out = true;
            if (c2[bf] > 0 && !mbar_wait_bounded(&S.d2_bar[bf], (c2[bf] - 1) & 1u, BTC_WAIT_LIMIT))
                timed_out = true;
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
    if (timed_out && lane == 0) set_status(P.hdr, UNIGS_ERR_TIMEOUT);
}

template <int NS>
static void launch_bwd_tc_t(const BwdTcParams& P, int grid, cudaStream_t st) {
    const size_t smem = sizeof(BwdTcSmem<NS>);
    ensure_smem_limit(reinterpret_cast<const void*>(&render_bwd_tc_kernel<NS>), (int)smem);
    render_bwd_tc_kernel<NS><<<grid, BTC_THREADS, smem, st>>>(P);
}

bool bwd_tc_selected(const unigs_plan& p) {
    return p.feat_dtype == 1 && p.n_sem >= 9 && p.n_sem <= UNIGS_MAX_SEM &&
           !(p.cfg.flags & UNIGS_FLAG_SIMT_LOGITS) &&
           (p.cfg.batch == 0 || p.cfg.batch == BTC_BATCH) &&
           (p.cfg.ctas_per_sm == 0 || p.cfg.ctas_per_sm == BTC_CTAS_PER_SM);
}

int launch_render_bwd_tc(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                         const unigs_outputs& fwd, const unigs_grad_outputs& go,
                         const unigs_param_grads& grads, double* grec, cudaStream_t st) {
    BwdTcParams P;
    P.tab = ws_ptr<CamTable>(ws, p, OFF_CAM);
    P.n_cams = p.n_cams;
    P.n_sem = p.n_sem;
    P.n = p.n;
    P.n_tiles = p.n_tiles;
    P.rec = ws_ptr<float>(ws, p, OFF_REC);
    P.sem = static_cast<const __nv_bfloat16*>(g.sem);
    P.vals = sorted_buffer(p) ? ws_ptr<uint32_t>(ws, p, OFF_VALS1)
                              : ws_ptr<uint32_t>(ws, p, OFF_VALS0);
    P.ranges = ws_ptr<uint2>(ws, p, OFF_RANGES);
    P.order = ws_ptr<uint32_t>(ws, p, OFF_ORDER);
    WsHeader* hdr = ws_ptr<WsHeader>(ws, p, OFF_HDR);
    P.work = &hdr->work_bwd;
    P.hdr = hdr;
    P.T_final = fwd.T_final;
    P.n_contrib = fwd.n_contrib;
    P.go = go;
    P.grec = grec;
    P.gsem = grads.sem;
    P.alpha_min = p.cfg.alpha_min;
    P.alpha_max = p.cfg.alpha_max;
    P.center_depth = (p.cfg.flags & UNIGS_FLAG_CENTER_DEPTH) ? 1 : 0;
    P.sem_bulk = ((p.n_sem * 2) % 16 == 0) && ((reinterpret_cast<uintptr_t>(P.sem) & 15) == 0);
    cudaMemsetAsync(P.work, 0, sizeof(uint32_t), st);
    int64_t grid = (int64_t)sm_count() * BTC_CTAS_PER_SM;
    if (grid > p.n_tiles) grid = p.n_tiles;
    if (p.n_sem <= 16)
        launch_bwd_tc_t<16>(P, (int)grid, st);
    else if (p.n_sem <= 32)
        launch_bwd_tc_t<32>(P, (int)grid, st);
    else
        launch_bwd_tc_t<64>(P, (int)grid, st);
    return 1;
}

}  // namespace unigs
