// Forward composite (Alg. 2) with the semantic blend of Eq. semantic_render
// on the 5th-generation tensor cores, for bfloat16 logit storage.
//
// Per tile and batch of B Gaussians the logit blend is a dense product:
// O[p][c] += sum_j W[p][j] F[j][c], with W[p][j] = alpha_j T_j at pixel p (0
// where Gaussian j is skipped, culled, or after the pixel's stop) and F the
// batch's logit rows.  Every other channel (RGB, depth, normal, k, T) and the
// per-pixel walk are those of the SIMT kernel (render_fwd.cu); only the 2C
// FMAs per blended pair move to the tensor core, which also frees the C
// per-pixel logit accumulators from the registers.
//
// Precision: F is exact in bfloat16 (the storage format).  W is split into
// bfloat16 hi + lo parts (w = hi + lo + r with |r| <= 2^-18 |w|), so two MMAs
// per K-step reproduce the float32 blend to ~4e-6 relative; products are exact
// and accumulate in float32 in tensor memory.
//
// Layout: the 256 pixels of the tile are two M = 128 tiles (thread tid owns
// row tid, i.e. tensor-memory lane tid % 128 of M-tile tid / 128); the
// accumulators of the tile live in 2 NS float32 tensor-memory columns for the
// whole tile list.  Operands are K-major without swizzle (8 x 16-byte core
// matrices): each thread zeroes its W rows (both splits) and stores the two
// parts of each weight it blends; the staged bfloat16 rows are transposed
// into F^T by the CTA.  After each batch one thread issues 2 x 2 x (B/16) MMAs of 128 x NS x 16
// and commits them to the mbarrier of that batch's operand buffer; operands
// are double-buffered, so a batch only waits for the MMAs of two batches back
// before it rewrites a buffer.  At the end of the tile every warp reads its 32
// lanes back with tcgen05.ld and writes the logits.
#include "launch.h"
#include "splat.cuh"
#include "tcgen05.cuh"

#include <type_traits>

namespace unigs {

constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

struct FwdTcParams {
    const CamTable* tab;
    int n_cams;
    int n_sem;
    int64_t n;
    int64_t n_tiles;
    const float* rec;
    const void* sem;           // rows [n][n_sem]: bfloat16, or float32 (F32 kernels)
    const uint32_t* vals;
    const uint2* ranges;
    const uint32_t* order;
    uint32_t* work;
    WsHeader* hdr;
    unigs_outputs out;
    float alpha_min, alpha_max, T_min;
    int center_depth;
    int sem_bulk;
};

template <int NS, int B, bool F32>
struct FwdTcSmem {
    using SemT = typename std::conditional<F32, float, __nv_bfloat16>::type;
    static constexpr int SPLITS_F = F32 ? 2 : 1;  // float32 features: bfloat16 hi + lo
    static constexpr int SBO = 16 * B;            // bytes between 8-row core-matrix groups
    static constexpr int W_BYTES = 128 * B * 2;   // one split of one M-tile
    static constexpr int F_BYTES = NS * B * 2;
    __align__(128) unsigned char wa[2][2][2][W_BYTES];       // [buffer][split][M-tile]
    __align__(128) unsigned char fb[2][SPLITS_F][F_BYTES];   // [buffer][split] F^T, NS x B
    __align__(16) float rec[2][B][REC_FLOATS];
    __align__(16) SemT semb[2][B][NS];
    uint64_t bar[2];
    uint64_t mma_bar[2];  // MMA completion per operand buffer
    uint32_t tmem_base;
    int tile;
    uint32_t issued[2];   // staging phases started per buffer (one thread counts)
};

template <int NS>
__host__ __device__ constexpr uint32_t tmem_cols() {
    return 2 * NS < 32 ? 32u : (uint32_t)(2 * NS);
}

template <int NS, int B, bool F32>
__device__ __forceinline__ void tc_issue_batch(const FwdTcParams& P, FwdTcSmem<NS, B, F32>& S,
                                               int buf, uint32_t first, int count, int cam) {
    using SemT = typename FwdTcSmem<NS, B, F32>::SemT;
    // executed by warp 0 only
    const int lane = threadIdx.x & 31;
    const uint32_t row_bytes = (uint32_t)(P.n_sem * sizeof(SemT));
    const uint32_t per = REC_FLOATS * 4 + (P.sem_bulk ? row_bytes : 0u);
    if (lane == 0) mbar_arrive_expect_tx(&S.bar[buf], per * (uint32_t)count);
    __syncwarp();
    for (int i = lane; i < count; i += 32) {
        const uint32_t g = P.vals[first + i];
        const size_t r = (size_t)cam * (size_t)P.n + g;
        bulk_g2s(&S.rec[buf][i][0], P.rec + r * REC_FLOATS, REC_FLOATS * 4, &S.bar[buf]);
        const SemT* src = static_cast<const SemT*>(P.sem) + (size_t)g * P.n_sem;
        if (P.sem_bulk)
            bulk_g2s(&S.semb[buf][i][0], src, row_bytes, &S.bar[buf]);
        else
            for (int c = 0; c < P.n_sem; ++c) S.semb[buf][i][c] = src[c];
    }
}

template <int NS, int B, bool F32>
// batch 16: 47 KB of shared memory and <= 64 registers, 4 CTAs per SM (4 x
// 128 accumulator columns fill the tensor memory); larger batches: 2
__global__ void __launch_bounds__(256, (B <= 16 ? 4 : 2)) render_fwd_tc_kernel(const FwdTcParams P) {
    using Sm = FwdTcSmem<NS, B, F32>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Sm& S = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    constexpr uint32_t NCOLS = tmem_cols<NS>();
    constexpr uint32_t IDESC = idesc_bf16_f32(128, NS);

    // once per CTA: zero the staging (rows shorter than NS stay zero-padded),
    // init barriers, allocate the accumulator columns
    for (int j = tid; j < 2 * B * NS; j += 256)
        (&S.semb[0][0][0])[j] = typename Sm::SemT(0.f);
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_init(&S.mma_bar[0], 1);
        mbar_init(&S.mma_bar[1], 1);
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

    // staging phases waited for per buffer (uniform across the CTA).  After a
    // bounded wait gave up, warp 0 (which waits on every phase itself) issues
    // no further copy, so at most one copy per buffer is ever in flight and
    // the exit drain below finds it by its count in S.issued.
    uint32_t loads[2] = {0u, 0u};
    // MMA commits and completed waits per operand buffer (uniform across the
    // CTA); each buffer's barrier is waited on before its next commit, so its
    // phases never run two ahead of the waits
    uint32_t commits0 = 0, commits1 = 0, waited0 = 0, waited1 = 0;
    bool timed_out = false;
    uint32_t n_eval = 0, n_blend = 0;
    const int mt = tid >> 7, row = tid & 127;
    const int wrow = (row >> 3) * Sm::SBO + (row & 7) * 16;
    uint32_t opbuf = 0;  // operand buffer of the next batch (alternates across tiles too)

    for (;;) {
        if (tid == 0) S.tile = (int)atomicAdd(P.work, 1u);
        __syncthreads();
        const int64_t t = S.tile;
        __syncthreads();
        if (t >= P.n_tiles) break;
        const int64_t gtile = P.order[t];
        int cam_idx;
        const DevCam& cam = cam_of_tile(P.tab, P.n_cams, gtile, &cam_idx);
        const int64_t ltile = gtile - cam.tile_off;
        const int tx = (int)(ltile % cam.tiles_x), ty = (int)(ltile / cam.tiles_x);
        int lx, ly;
        const int tw = cam.tile_w, th = cam.tile_h;
        tile_pixel(tid, tw, &lx, &ly);
        const int u = tx * tw + lx, v = ty * th + ly;
        // the warp's 8x4 pixel block, for the per-warp bounding-box skip
        int wbx, wby;
        warp_block(warp, tw, &wbx, &wby);
        const float bx0 = (float)(tx * tw + wbx);
        const float by0 = (float)(ty * th + wby);
        const bool inside = u < cam.width && v < cam.height;
        const float uf = (float)u, vf = (float)v;
        const float xt = (uf - cam.cx) / cam.fx, yt = (vf - cam.cy) / cam.fy;

        const uint2 range = P.ranges[gtile];
        const int n_items = (int)(range.y - range.x);
        const int n_batches = (n_items + B - 1) / B;
        if (warp == 0 && n_batches > 0 && !__any_sync(0xffffffffu, timed_out)) {
            tc_issue_batch<NS, B, F32>(P, S, 0, range.x, min(B, n_items), cam_idx);
            if ((tid & 31) == 0) ++S.issued[0];
        }
        __syncthreads();

        float T = 1.f;
        float crgb[3] = {0.f, 0.f, 0.f}, cdep = 0.f, cn[3] = {0.f, 0.f, 0.f}, ck = 0.f;
        uint32_t last = 0;
        bool done = !inside;
        int batches_done = 0;

        for (int b = 0; b < n_batches; ++b) {
            const int buf = b & 1;
            if (warp == 0 && b + 1 < n_batches && !__any_sync(0xffffffffu, timed_out)) {
                tc_issue_batch<NS, B, F32>(P, S, buf ^ 1, range.x + (b + 1) * B,
                                      min(B, n_items - (b + 1) * B), cam_idx);
                if ((tid & 31) == 0) ++S.issued[buf ^ 1];
            }
            if (!mbar_wait_bounded(&S.bar[buf], loads[buf] & 1u, TC_WAIT_LIMIT)) timed_out = true;
            ++loads[buf];
            // the MMAs that last read this operand buffer (two batches back)
            // must be complete before it is rewritten
            const int ob = (int)opbuf;
            {
                const uint32_t cm = ob ? commits1 : commits0;
                if ((ob ? waited1 : waited0) < cm) {
                    if (!mbar_wait_bounded(&S.mma_bar[ob], (cm - 1) & 1u, TC_WAIT_LIMIT))
                        timed_out = true;
                    if (ob) waited1 = cm; else waited0 = cm;
                }
            }
            const int count = min(B, n_items - b * B);
            // F^T: channel c, Gaussians 8 jc .. 8 jc + 7 as one 16-byte core row
            // (float32 features: the bfloat16 hi part and the bfloat16 rounding
            // of the remainder, f = hi + lo + r with |r| <= 2^-18 |f|)
            for (int task = tid; task < NS * (B / 8); task += 256) {
                const int c = task / (B / 8), jc = task % (B / 8);
                const int off = (c >> 3) * Sm::SBO + jc * 128 + (c & 7) * 16;
                if (F32) {
                    const float* col = reinterpret_cast<const float*>(&S.semb[buf][0][0]) + c;
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float f0 = col[(8 * jc + 2 * e) * NS];
                        const float f1 = col[(8 * jc + 2 * e + 1) * NS];
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(f0);
                        const __nv_bfloat16 h1 = __float2bfloat16_rn(f1);
                        h[e] = (uint32_t)__bfloat16_as_ushort(h0) |
                               ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                        l[e] = (uint32_t)__bfloat16_as_ushort(
                                   __float2bfloat16_rn(f0 - __bfloat162float(h0))) |
                               ((uint32_t)__bfloat16_as_ushort(
                                    __float2bfloat16_rn(f1 - __bfloat162float(h1)))
                                << 16);
                    }
                    *reinterpret_cast<uint4*>(&S.fb[ob][0][0] + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(&S.fb[ob][F32 ? 1 : 0][0] + off) =
                        make_uint4(l[0], l[1], l[2], l[3]);
                } else {
                    const unsigned short* col =
                        reinterpret_cast<const unsigned short*>(&S.semb[buf][0][0]) + c;
                    uint4 q;
                    q.x = (uint32_t)col[(8 * jc + 0) * NS] | ((uint32_t)col[(8 * jc + 1) * NS] << 16);
                    q.y = (uint32_t)col[(8 * jc + 2) * NS] | ((uint32_t)col[(8 * jc + 3) * NS] << 16);
                    q.z = (uint32_t)col[(8 * jc + 4) * NS] | ((uint32_t)col[(8 * jc + 5) * NS] << 16);
                    q.w = (uint32_t)col[(8 * jc + 6) * NS] | ((uint32_t)col[(8 * jc + 7) * NS] << 16);
                    *reinterpret_cast<uint4*>(&S.fb[ob][0][0] + off) = q;
                }
            }
            const bool skip = __all_sync(0xffffffffu, done || timed_out);
            // this thread's W rows: zero, then the weights of the Gaussians it
            // blends (hi and lo bfloat16 parts)
            unsigned char* w0 = &S.wa[ob][0][mt][0] + wrow;
            unsigned char* w1 = &S.wa[ob][1][mt][0] + wrow;
#pragma unroll
            for (int jc = 0; jc < B / 8; ++jc) {
                *reinterpret_cast<uint4*>(w0 + jc * 128) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(w1 + jc * 128) = make_uint4(0u, 0u, 0u, 0u);
            }
            if (!skip) {
#pragma unroll 1
                for (int j = 0; j < count; ++j) {
                    const float* rc = &S.rec[buf][j][0];
                    if (warp_block_misses(rc, bx0, by0)) continue;  // uniform per warp
                    if (done) continue;
                    float dx, dy, Gs;
                    float wq;
                    const float alpha = splat_alpha(rc, uf, vf, P.alpha_max, &dx, &dy, &Gs, &wq);
                    ++n_eval;
                    if (alpha < P.alpha_min) continue;
                    const float test_T = T * (1.f - alpha);
                    if (test_T < P.T_min) {
                        done = true;
                        continue;
                    }
                    ++n_blend;
                    const float w = alpha * T;
                    PairGeom G;
                    pair_geometry(rc, xt, yt, dx, dy, G);
                    const float depth = P.center_depth ? rc[R_Z] : G.t;
                    const float nsg = (G.inside ? -G.inv_m : G.inv_m) * w;
                    crgb[0] = fmaf(w, rc[R_RGB], crgb[0]);
                    crgb[1] = fmaf(w, rc[R_RGB + 1], crgb[1]);
                    crgb[2] = fmaf(w, rc[R_RGB + 2], crgb[2]);
                    cdep = fmaf(w, depth, cdep);
                    cn[0] = fmaf(nsg, G.m[0], cn[0]);
                    cn[1] = fmaf(nsg, G.m[1], cn[1]);
                    cn[2] = fmaf(nsg, G.m[2], cn[2]);
                    ck = fmaf(w, rc[R_K], ck);
                    T = test_T;
                    last = (uint32_t)(b * B + j + 1);
                    // w = hi + lo, both bfloat16
                    const __nv_bfloat16 wh = __float2bfloat16_rn(w);
                    const int off = (j >> 3) * 128 + (j & 7) * 2;
                    *reinterpret_cast<__nv_bfloat16*>(w0 + off) = wh;
                    *reinterpret_cast<__nv_bfloat16*>(w1 + off) =
                        __float2bfloat16_rn(w - __bfloat162float(wh));
                }
            }
            fence_async_shared();
            const int alive = __syncthreads_count(!done && !timed_out);
            // one thread issues the batch's MMAs: per M-tile and K-step, W_hi F_hi
            // and W_lo F_hi, plus W_hi F_lo for float32 features (W_lo F_lo is
            // below the float32 rounding of the sum)
            if (tid == 0) {
                tc_fence_after_sync();
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const uint32_t d = tmem + (uint32_t)(m * NS);
#pragma unroll
                    for (int pr = 0; pr < (F32 ? 3 : 2); ++pr) {
                        const int sw = pr == 1 ? 1 : 0, sf = pr == 2 ? 1 : 0;
#pragma unroll
                        for (int s = 0; s < B / 16; ++s) {
                            const uint64_t a = smem_desc_kmajor(&S.wa[ob][sw][m][0] + s * 256,
                                                                128, Sm::SBO);
                            const uint64_t f =
                                smem_desc_kmajor(&S.fb[ob][sf][0] + s * 256, 128, Sm::SBO);
                            const uint32_t acc = (batches_done > 0 || pr > 0 || s > 0) ? 1u : 0u;
                            mma_bf16(d, a, f, IDESC, acc);
                        }
                    }
                }
                mma_commit(&S.mma_bar[ob]);
            }
            if (ob) ++commits1; else ++commits0;
            opbuf ^= 1u;
            ++batches_done;
            if (alive == 0) {
                if (b + 1 < n_batches) {
                    if (!mbar_wait_bounded(&S.bar[buf ^ 1], loads[buf ^ 1] & 1u, TC_WAIT_LIMIT))
                        timed_out = true;
                    ++loads[buf ^ 1];
                }
                break;
            }
        }
        // logits: the accumulators of this thread's row (zero without a batch)
        if (waited0 < commits0) {
            if (!mbar_wait_bounded(&S.mma_bar[0], (commits0 - 1) & 1u, TC_WAIT_LIMIT))
                timed_out = true;
            waited0 = commits0;
        }
        if (waited1 < commits1) {
            if (!mbar_wait_bounded(&S.mma_bar[1], (commits1 - 1) & 1u, TC_WAIT_LIMIT))
                timed_out = true;
            waited1 = commits1;
        }
        tc_fence_after_sync();
        const int W = cam.width;
        const int64_t HW = (int64_t)cam.height * W;
        const int64_t pix = cam.pix_off;
        const int64_t idx = (int64_t)v * W + u;
        float* lo_out = P.out.logits + pix * (int64_t)P.n_sem + idx;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll
        for (int ch = 0; ch < NS / 16; ++ch) {
            float o[16];
            if (batches_done > 0) {
                tmem_ld16(tmem + lane_base + (uint32_t)((warp >> 2) * NS + 16 * ch), o);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) o[i] = 0.f;
            }
            if (inside)
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (16 * ch + i < P.n_sem) lo_out[(int64_t)(16 * ch + i) * HW] = o[i];
        }
        tc_fence_before_sync();
        if (inside) {
            P.out.rgb[pix * 3 + 0 * HW + idx] = crgb[0];
            P.out.rgb[pix * 3 + 1 * HW + idx] = crgb[1];
            P.out.rgb[pix * 3 + 2 * HW + idx] = crgb[2];
            P.out.depth[pix + idx] = cdep;
            P.out.normal_g[pix * 3 + 0 * HW + idx] = cn[0];
            P.out.normal_g[pix * 3 + 1 * HW + idx] = cn[1];
            P.out.normal_g[pix * 3 + 2 * HW + idx] = cn[2];
            P.out.kmap[pix + idx] = ck;
            P.out.T_final[pix + idx] = T;
            P.out.n_contrib[pix + idx] = last;
        }
        if (__syncthreads_or(timed_out)) break;
    }
    // Before the CTA exits: no bulk copy may still be landing in its shared
    // memory, and no MMA may still be writing its tensor-memory columns (each
    // tile waits for its last commits; after a timeout the last commit of each
    // operand buffer is waited for once more, bounded).  Then the columns are
    // returned: a CTA frees its tensor memory before it exits, also when a
    // wait gave up.
    if (tid == 0 && !drain_bulk(S.bar, S.issued[0], S.issued[1], TC_WAIT_LIMIT)) timed_out = true;
    if (commits0 > 0 && !mbar_wait_bounded(&S.mma_bar[0], (commits0 - 1) & 1u, TC_WAIT_LIMIT))
        timed_out = true;
    if (commits1 > 0 && !mbar_wait_bounded(&S.mma_bar[1], (commits1 - 1) & 1u, TC_WAIT_LIMIT))
        timed_out = true;
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
    if (timed_out && (tid & 31) == 0) set_status(P.hdr, UNIGS_ERR_TIMEOUT);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
        n_blend += __shfl_xor_sync(0xffffffffu, n_blend, o);
    }
    if ((tid & 31) == 0 && n_eval) {
        atomicAdd(&P.hdr->n_eval, (unsigned long long)n_eval);
        atomicAdd(&P.hdr->n_blend, (unsigned long long)n_blend);
    }
}

template <int NS, int B, bool F32>
static void launch_fwd_tc_t(const FwdTcParams& P, int grid, cudaStream_t st) {
    const size_t smem = sizeof(FwdTcSmem<NS, B, F32>);
    // per device; a failure surfaces as the launch error the entry point returns
    ensure_smem_limit(reinterpret_cast<const void*>(&render_fwd_tc_kernel<NS, B, F32>), (int)smem);
    render_fwd_tc_kernel<NS, B, F32><<<grid, 256, smem, st>>>(P);
}

template <int B, bool F32>
static void launch_fwd_tc_b(const FwdTcParams& P, int grid, cudaStream_t st) {
    if (P.n_sem <= 16)
        launch_fwd_tc_t<16, B, F32>(P, grid, st);
    else if (P.n_sem <= 32)
        launch_fwd_tc_t<32, B, F32>(P, grid, st);
    else
        launch_fwd_tc_t<64, B, F32>(P, grid, st);
}

template <bool F32>
static void launch_fwd_tc_f(const FwdTcParams& P, int batch, int grid, cudaStream_t st) {
    switch (batch) {
        case 16: launch_fwd_tc_b<16, F32>(P, grid, st); break;
        case 64: launch_fwd_tc_b<64, F32>(P, grid, st); break;
        default: launch_fwd_tc_b<32, F32>(P, grid, st); break;
    }
}

static bool fwd_tc_plan(const unigs_plan& p) {
    return p.n_sem >= 9 && p.n_sem <= UNIGS_MAX_SEM && !(p.cfg.flags & UNIGS_FLAG_SIMT_LOGITS);
}

bool fwd_tc_eligible(const unigs_plan& p, const unigs_gaussians& g) {
    return fwd_tc_plan(p) && g.sem != nullptr;
}

bool sem32_needed(const unigs_plan& p) {
    if (!p.feat_dtype || p.n_sem <= 0 || p.n <= 0) return false;
    return !(fwd_tc_plan(p) && bwd_tc_selected(p));
}

int launch_render_fwd_tc(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                         const unigs_outputs& out, cudaStream_t st) {
    if (p.n_tiles == 0) return 0;
    FwdTcParams P;
    P.tab = ws_ptr<CamTable>(ws, p, OFF_CAM);
    P.n_cams = p.n_cams;
    P.n_sem = p.n_sem;
    P.n = p.n;
    P.n_tiles = p.n_tiles;
    P.rec = ws_ptr<float>(ws, p, OFF_REC);
    P.sem = g.sem;
    P.vals = sorted_buffer(p) ? ws_ptr<uint32_t>(ws, p, OFF_VALS1) : ws_ptr<uint32_t>(ws, p, OFF_VALS0);
    P.ranges = ws_ptr<uint2>(ws, p, OFF_RANGES);
    P.order = ws_ptr<uint32_t>(ws, p, OFF_ORDER);
    WsHeader* hdr = ws_ptr<WsHeader>(ws, p, OFF_HDR);
    P.work = &hdr->work_fwd;
    P.hdr = hdr;
    P.out = out;
    P.alpha_min = p.cfg.alpha_min;
    P.alpha_max = p.cfg.alpha_max;
    P.T_min = p.cfg.T_min;
    P.center_depth = (p.cfg.flags & UNIGS_FLAG_CENTER_DEPTH) ? 1 : 0;
    const int esz = p.feat_dtype ? 2 : 4;
    P.sem_bulk = ((p.n_sem * esz) % 16 == 0) && ((reinterpret_cast<uintptr_t>(P.sem) & 15) == 0);
    cudaMemsetAsync(P.work, 0, sizeof(uint32_t), st);
    // defaults: batch 16, 4 CTAs per SM; at most 4 CTAs per SM hold
    // accumulator columns at once (512 per SM)
    const int batch = p.cfg.batch_fwd > 0 ? p.cfg.batch_fwd : 16;
    int ctas = p.cfg.ctas_per_sm_fwd > 0 ? p.cfg.ctas_per_sm_fwd : 4;
    if (ctas > 4) ctas = 4;
    int64_t grid = (int64_t)sm_count() * ctas;
    if (grid > p.n_tiles) grid = p.n_tiles;
    if (p.feat_dtype)
        launch_fwd_tc_f<false>(P, batch, (int)grid, st);
    else
        launch_fwd_tc_f<true>(P, batch, (int)grid, st);
    return 1;
}

}  // namespace unigs
