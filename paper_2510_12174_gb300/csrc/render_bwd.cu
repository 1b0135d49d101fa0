// Backward composite (Alg. 4) and preprocess backward.
//
// Kernel 1, persistent CTAs pulling 16x16 tiles longest list first, one pixel
// per thread: each pixel restores T = T_final and walks its list backwards
// from the last blended Gaussian, T <- T / (1 - alpha_i),
// w_i = alpha_i T_i.  With G_i = sum_ch g_ch x_i,ch (upstream gradient dotted
// with the Gaussian's features) and S_i = sum_{j>i} w_j G_j,
//   dL/dx_i,ch = w_i g_ch            (Eq. gradiento, Eq. gradientk)
//   dL/dalpha_i = T_i G_i - S_i / (1 - alpha_i).
// The feature gradients of the depth (t_mid, supplement Sec. 2:
// dt/db = -1/2a, dt/da = b/2a^2 with b = 2 v_s.d_s) and of the ellipsoid
// normal flow to the per-(camera, Gaussian) ray-ellipsoid setup (M_c, v_s,
// N_w); dL/dalpha flows to opacity, conic and projected centre.  The 32
// lanes of a warp (32 pixels) are summed with a butterfly transpose-reduction
// (lane L ends with component L) before one float32 atomic per lane.  The
// semantic gradients sum_l w_l g_O,l of the warp's 32 pixels are gathered
// densely from the tile's upstream-gradient rows in shared memory (4 channels
// per 16-byte load, w = 0 for pixels that do not contribute), one 16-byte
// atomic per 4 channels.
//
// Kernel 2, one thread per Gaussian, loops over the cameras: conic -> 2D
// covariance -> (J, Sigma) -> mean, rotation, scale (EWA chain of 3DGS);
// M_c = S^-1 R^T R_cw, v_s = S^-1 R^T (C - mu), N_w = R S^-1 -> R, s, mu
// (supplement Sec. 2: dL/ds_k = -(g_vs,k v_s,k + g_ds,k d_s,k)/s_k per ray,
// dL/dmu = -R (g_vs / s)); colour -> SH coefficients and viewing direction;
// then R(q^) -> q^ -> q through the tangent projection (I - q^ q^T)/|q|.
#include <type_traits>

#include "launch.h"
#include "sh.cuh"
#include "bwd_pair.cuh"

namespace unigs {

constexpr uint32_t BWAIT_LIMIT = 1u << 22;


struct BwdParams {
    const CamTable* tab;
    int n_cams;
    int n_sem;
    int64_t n;
    int64_t n_tiles;
    const float* rec;
    const float* sem;          // float32 rows (a float32 copy for bfloat16 storage)
    const uint32_t* vals;
    const uint2* ranges;
    const uint32_t* order;     // global tile ids, longest list first
    uint32_t* work;            // tile counter
    WsHeader* hdr;
    const float* T_final;
    const uint32_t* n_contrib;
    unigs_grad_outputs go;
    double* grec;              // float64 accumulators (see the RED below)
    float* gsem;
    float alpha_min, alpha_max;
    int center_depth;
    int sem_bulk;
};

template <int NS, int B>
struct BwdSmem {
    // dL/dlogits of the tile's pixels, one row of NS floats per thread; the
    // 16-byte chunk k of row p is stored at chunk k ^ (p % (NS / 4)), so both
    // the per-thread row reads and the per-row channel gathers of a warp are
    // free of bank conflicts without padding
    float rec[2][B][REC_FLOATS];
    float sem[2][B][NS];
    float gO[TILE_PIX * NS];
    float2 wv[8][32];  // per warp: (w, w) of its pixels for the current Gaussian
    uint32_t ids[2][B];
    uint64_t bar[2];   // batch staged (bulk bytes + the producer warp's arrival)
    uint64_t cons[2];  // batch consumed (one arrival per warp)
    uint32_t max_last;
    int tile;
    uint32_t issued[2];  // staging phases started per buffer (one thread counts)
};

// Offset of channel c of pixel row p in the swizzled upstream-gradient tile.
template <int NS>
__device__ __forceinline__ int go_index(int p, int c) {
    return p * NS + ((((c >> 2) ^ p) & (NS / 4 - 1)) << 2) + (c & 3);
}

// f(integral_constant<int, I>) for I = 0 .. N-1, unrolled at compile time.
template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// 16-byte shared-memory load at a 32-bit shared address plus a constant.
template <int OFF>
__device__ __forceinline__ float4 lds128(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr), "n"(OFF));
    return v;
}

// Shared address of chunk 0 of upstream-gradient row p with the row's swizzle
// key folded in: the tile and its rows (NS floats) are aligned to the row
// size, so chunk c of the row is at go_row(p) ^ (16 c).
template <int NS>
__device__ __forceinline__ uint32_t go_row(uint32_t go_base, int p) {
    return (go_base + (uint32_t)(p * NS * 4)) | ((uint32_t)(p & (NS / 4 - 1)) << 4);
}

// dot(gO row, semantic row) with 16-byte shared-memory loads and packed
// float32 FMAs (four partial sums, one per channel residue mod 4); a_row from
// go_row.
template <int NS>
__device__ __forceinline__ float sem_dot(uint32_t a_row, const float* row) {
    float2 acc01 = make_float2(0.f, 0.f), acc23 = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < NS / 4; ++c) {
        const float4 a = lds128<0>(a_row ^ (uint32_t)(c << 4));
        const float4 b = reinterpret_cast<const float4*>(row)[c];
        acc01 = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), acc01);
        acc23 = __ffma2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w), acc23);
    }
    return (acc01.x + acc23.x) + (acc01.y + acc23.y);
}
template <int NS, int B>
__device__ __forceinline__ void bwd_issue(const BwdParams& P, BwdSmem<NS, B>& S, int buf,
                                          uint32_t first, int count, int cam) {
    const int lane = threadIdx.x & 31;
    const uint32_t row_bytes = (uint32_t)(P.n_sem * sizeof(float));
    const uint32_t per = REC_FLOATS * 4 + (P.sem_bulk ? row_bytes : 0u);
    if (lane == 0) mbar_expect_tx(&S.bar[buf], per * (uint32_t)count);
    __syncwarp();
    for (int i = lane; i < count; i += 32) {
        const uint32_t g = P.vals[first + i];
        S.ids[buf][i] = g;
        const size_t r = (size_t)cam * (size_t)P.n + g;
        bulk_g2s(&S.rec[buf][i][0], P.rec + r * REC_FLOATS, REC_FLOATS * 4, &S.bar[buf]);
        if (P.n_sem > 0) {
            const float* src = P.sem + (size_t)g * P.n_sem;
            if (P.sem_bulk)
                bulk_g2s(&S.sem[buf][i][0], src, row_bytes, &S.bar[buf]);
            else
                for (int c = 0; c < P.n_sem; ++c) S.sem[buf][i][c] = src[c];
        }
    }
    // the warp's plain stores (ids, unaligned rows) are released by the
    // producer's arrival, which the consumers' wait acquires
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.bar[buf]);
}

template <int NS, int B>
// batch 8 (73 KB of shared memory at 64 logits): 3 CTAs per SM, 80 registers;
// larger batches (80 KB at 16, 94 KB at 32): 2 CTAs per SM, 128 registers
__global__ void __launch_bounds__(256, (B <= 8 ? 3 : 2)) render_bwd_kernel(const BwdParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BwdSmem<NS, B>& S = *reinterpret_cast<BwdSmem<NS, B>*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // once per CTA: init barriers, zero the semantic padding
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_init(&S.cons[0], 8);
        mbar_init(&S.cons[1], 8);
        fence_mbar_init();
        S.issued[0] = S.issued[1] = 0u;
    }
    for (int j = tid; j < 2 * B * NS; j += 256) (&S.sem[0][0][0])[j] = 0.f;
    // the upstream-gradient rows are addressed by XOR within a row, which
    // needs the tile aligned to the row size (it sits at a multiple of 256
    // bytes of the dynamic shared memory, whose start is so aligned)
    const uint32_t go_base = smem_u32(S.gO);
    if (go_base & (uint32_t)(NS * 4 - 1)) {
        if (tid == 0) set_status(P.hdr, UNIGS_ERR_CUDA);
        return;
    }
    const uint32_t a_row = go_row<NS>(go_base, tid);
    __syncthreads();
    // per buffer: phases of bar[] waited for and consumptions (uniform across
    // the CTA); scalars, so that they stay in registers
    uint32_t loads0 = 0u, loads1 = 0u, used0 = 0u, used1 = 0u;
    bool timed_out = false;

    for (;;) {
        if (tid == 0) {
            S.tile = (int)atomicAdd(P.work, 1u);
            S.max_last = 0;
        }
        __syncthreads();
        const int64_t t = S.tile;
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
        const int W = cam.width;
        const int64_t HW = (int64_t)cam.height * W;
        const int64_t pix = cam.pix_off;
        const int64_t idx = (int64_t)v * W + u;

        float T = 1.f;
        uint32_t last = 0;
        PixelUp up = {{0.f, 0.f, 0.f}, 0.f, {0.f, 0.f, 0.f}, 0.f};
        // upstream logit gradients of this pixel -> shared memory row tid (zero
        // padded), read by this thread for G_i and by the warp's channel gather
#pragma unroll 8
        for (int c = 0; c < NS; ++c)
            S.gO[go_index<NS>(tid, c)] = (inside && P.go.logits && c < P.n_sem)
                               ? P.go.logits[pix * (int64_t)P.n_sem + c * HW + idx] : 0.f;
        if (inside) {
            T = P.T_final[pix + idx];
            last = P.n_contrib[pix + idx];
            load_pixel_up(P.go, pix, HW, idx, up);
        }
        if (last) atomicMax(&S.max_last, last);
        // the warp's own last list position: Gaussians behind it are skipped
        // by the whole warp
        const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);
        __syncthreads();
        const int n_items = (int)S.max_last;
        const int n_batches = (n_items + B - 1) / B;
        const uint2 range = P.ranges[gtile];
        // Staging pipeline: warp 0 stages batch it+1 while every warp composites
        // batch it; a buffer is restaged only after all 8 warps have arrived on
        // its "consumed" barrier, so the warps never meet at a CTA barrier
        // inside the tile.
        // Warp 0 restages a buffer only if none of its own waits gave up (a
        // warp-uniform decision): it waits on every staging phase itself, so
        // the buffer's previous copy was seen to land and at most one copy
        // per buffer is ever in flight; the exit drain finds it by S.issued.
        auto produce = [&](int bf, uint32_t first, int cnt) {
            const uint32_t u = bf ? used1 : used0;
            if (u > 0 && !mbar_wait_bounded(&S.cons[bf], (u - 1) & 1u, BWAIT_LIMIT))
                timed_out = true;
            if (__any_sync(0xffffffffu, timed_out)) return;
            bwd_issue<NS, B>(P, S, bf, first, cnt, cam_idx);
            if (lane == 0) ++S.issued[bf];
        };
        if (warp == 0 && n_batches > 0)
            produce(0, range.x + (n_batches - 1) * B, min(B, n_items - (n_batches - 1) * B));

        float Sacc = 0.f;  // sum over already processed (later) Gaussians of w_j G_j
        for (int it = 0; it < n_batches; ++it) {
            const int b = n_batches - 1 - it;
            const int buf = it & 1;
            if (warp == 0 && b > 0) produce(buf ^ 1, range.x + (b - 1) * B, B);
            {
                const uint32_t ph = buf ? loads1 : loads0;
                if (!mbar_wait_bounded(&S.bar[buf], ph & 1u, BWAIT_LIMIT)) timed_out = true;
                if (buf) ++loads1; else ++loads0;
            }
            const int count = min(B, n_items - b * B);
            if (!__all_sync(0xffffffffu, timed_out) && (uint32_t)(b * B) < wlast) {
            for (int j = min(count, (int)(wlast - (uint32_t)(b * B))) - 1; j >= 0; --j) {
                const uint32_t pos = (uint32_t)(b * B + j);
                const float* rc = &S.rec[buf][j][0];
                if (warp_block_misses(rc, bx0, by0)) continue;  // uniform per warp
                // alpha of every lane; the warp runs the pair's gradient only if
                // some lane contributes, and then as a whole: a lane that does not
                // contribute carries w = 0 and dL/dalpha = 0, which makes every
                // entry of its gradient vector zero (all intermediates are finite)
                float dx, dy, Gs, wq;
                const float alpha = splat_alpha(rc, uf, vf, P.alpha_max, &dx, &dy, &Gs, &wq);
                const bool contrib = !timed_out && pos < last && alpha >= P.alpha_min;
                if (!__any_sync(0xffffffffu, contrib)) continue;
                float gv[32];
                const float w = bwd_pair(rc, up, xt, yt, wq, dx, dy, alpha, Gs, contrib,
                                         sem_dot<NS>(a_row, &S.sem[buf][j][0]), P.alpha_max,
                                         P.center_depth, T, Sacc, gv);
                {
                    const uint32_t g = S.ids[buf][j];
                    const size_t rix = (size_t)cam_idx * (size_t)P.n + g;
                    // the warp's sum of component `lane`, added in float64: a
                    // Gaussian's record sums thousands of pixel terms that can
                    // cancel (near-camera, elongated splats), and a float32
                    // sum in atomic order would leave it off by the rounding
                    // of the partial sums, differently on every run
                    const float tot = warp_reduce_transpose32(gv, lane);
                    if (tot != 0.f) atomicAdd(P.grec + rix * GREC_FLOATS + lane, (double)tot);
                    if (P.n_sem > 0) {
                        // dL/do_j[c] = sum over the contributing pixels l of w_l gO_l[c]
                        {
                            // every row of the warp (w = 0 where the pixel does not
                            // contribute), NS/4 lanes per row (16-byte loads of 4
                            // channels), 128/NS rows per step; the lanes that share
                            // channels are then added.  Cheaper than looping over the
                            // contributing lanes only: most warps have many.
                            constexpr int LPR = NS / 4, RPS = 32 / LPR;
                            // w is stored twice so one 8-byte load gives the
                            // packed FMAs their operand pair
                            S.wv[warp][lane] = make_float2(w, w);
                            __syncwarp();
                            const int h = lane / LPR, c4 = lane % LPR;
                            // row r = i RPS + h holds channel chunk c4 at chunk
                            // c4 ^ (h % LPR) ^ ((i RPS) % LPR): the first part is
                            // folded into the lane's base address, the second
                            // repeats with i and is a constant
                            const uint32_t a_g =
                                (go_base + (uint32_t)((warp * 32 + h) * NS * 4)) |
                                ((uint32_t)(c4 ^ (h & (LPR - 1))) << 4);
                            float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
                            static_for<0, LPR>([&](auto ic) {
                                constexpr int i = decltype(ic)::value;
                                const float2 wr = S.wv[warp][i * RPS + h];
                                const float4 go = lds128<i * RPS * NS * 4>(
                                    a_g ^ (uint32_t)(((i * RPS) & (LPR - 1)) << 4));
                                a01 = __ffma2_rn(wr, make_float2(go.x, go.y), a01);
                                a23 = __ffma2_rn(wr, make_float2(go.z, go.w), a23);
                            });
#pragma unroll
                            for (int o = LPR; o < 32; o <<= 1) {
                                a01 = __fadd2_rn(a01, make_float2(
                                    __shfl_xor_sync(0xffffffffu, a01.x, o),
                                    __shfl_xor_sync(0xffffffffu, a01.y, o)));
                                a23 = __fadd2_rn(a23, make_float2(
                                    __shfl_xor_sync(0xffffffffu, a23.x, o),
                                    __shfl_xor_sync(0xffffffffu, a23.y, o)));
                            }
                            const float4 acc = make_float4(a01.x, a01.y, a23.x, a23.y);
                            __syncwarp();
                            const int c = 4 * c4;
                            if (h == 0 && c < P.n_sem) {
                                float* dst = P.gsem + (size_t)g * P.n_sem + c;
                                if ((P.n_sem & 3) == 0) {
                                    atomicAdd(reinterpret_cast<float4*>(dst), acc);
                                } else {
                                    const float av[4] = {acc.x, acc.y, acc.z, acc.w};
                                    for (int e = 0; e < 4 && c + e < P.n_sem; ++e)
                                        atomicAdd(dst + e, av[e]);
                                }
                            }
                        }
                    }
                }
            }
            }
            // this warp is done with the batch's buffers
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.cons[buf]);
            if (buf) ++used1; else ++used0;
        }
        // a bounded wait that gave up ends the CTA (uniformly)
        if (__syncthreads_or(timed_out)) break;
    }
    // no bulk copy may still be landing in this CTA's shared memory when it
    // exits (after a timeout at most one per buffer is in flight)
    if (tid == 0 && !drain_bulk(S.bar, S.issued[0], S.issued[1], BWAIT_LIMIT)) timed_out = true;
    if (timed_out && lane == 0) set_status(P.hdr, UNIGS_ERR_TIMEOUT);
}

// ------------------------------------------------------ record zeroing
// Zeroes the gradient record (GREC_FLOATS doubles) of every (camera,
// Gaussian) pair with a kept tile.  A warp reads 32 consecutive touched
// counts, then clears the flagged records two at a time, one 16-byte store
// per lane, so that each store instruction covers two whole records.
__global__ void __launch_bounds__(256)
    grec_zero_kernel(const uint32_t* __restrict__ touched, double2* __restrict__ grec,
                     int64_t total) {
    constexpr int PER = GREC_FLOATS / 2;  // 16-byte chunks per record
    static_assert(PER == 16, "two records per warp-wide store");
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31;
         base < total; base += stride) {
        const int64_t t = base + lane;
        uint32_t mask = __ballot_sync(0xffffffffu, t < total && touched[t] != 0);
        while (mask) {
            const int r0 = __ffs(mask) - 1;
            mask &= mask - 1;
            int r1 = -1;
            if (mask) {
                r1 = __ffs(mask) - 1;
                mask &= mask - 1;
            }
            const int r = lane < PER ? r0 : r1;
            if (r >= 0) grec[(base + r) * PER + (lane & (PER - 1))] = make_double2(0.0, 0.0);
        }
    }
}

// ---------------------------------------------------------------- kernel 2
struct PreBwdParams {
    const CamTable* tab;
    int n_cams;
    unigs_gaussians g;
    const float* rec;
    const double* grec;
    const float4* vp;          // e1^T V per (camera, Gaussian), from the preprocess
    const uint32_t* touched;
    unigs_param_grads out;
    float lowpass;
};

// Threads per block of the preprocess backward (4 warps).
constexpr int PREBWD_THREADS = 128;

// The preprocess backward works warp by warp on 32 Gaussians.  Their
// (camera, Gaussian) pairs with a kept tile are dealt to the warp's lanes 32
// at a time, so that no lane idles on a camera that does not see its
// Gaussian (about a third of the pairs have a kept tile); each pair's
// contributions are added to the Gaussian's row of shared-memory
// accumulators, which the Gaussian's own lane then maps onto the parameters.
// DEG is the SH degree: with the basis size a compile-time constant the
// basis, its gradient and the coefficient gradients are registers.  Four
// blocks per SM (a few spilled registers at degree 3) measured faster than
// three without spills.
template <int DEG>
__global__ void __launch_bounds__(PREBWD_THREADS, 4) preprocess_bwd_kernel(const PreBwdParams P) {
    constexpr int n_sh = (DEG + 1) * (DEG + 1);
    // accumulators per Gaussian: g_mu 3, g_R 9, g_s 3, g_th 3, g_op, g_k, g_sh
    constexpr int NACC = 20 + 3 * n_sh;
    constexpr int ACCS = NACC | 1;  // odd row stride: the lanes' rows start in different banks
    constexpr int WARPS = PREBWD_THREADS / 32;
    __shared__ float acc_all[WARPS][32 * ACCS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* acc = acc_all[wib];
    const int64_t n = P.g.n;
    const int64_t stride = (int64_t)gridDim.x * WARPS * 32;
    for (int64_t g0 = ((int64_t)blockIdx.x * WARPS + wib) * 32; g0 < n; g0 += stride) {
        // the cameras with a kept tile of this lane's Gaussian
        const int64_t own = g0 + lane;
        uint64_t mask = 0;
        if (own < n)
            for (int k = 0; k < P.n_cams; ++k)
                if (P.touched[(size_t)k * (size_t)n + (size_t)own]) mask |= 1ull << k;
        for (int e = lane; e < 32 * ACCS; e += 32) acc[e] = 0.f;
        const int cnt = __popcll(mask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int pre = incl - cnt;  // the lane's first pair in the warp's numbering
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
        for (int r0 = 0; r0 < total; r0 += 32) {
            const int q = r0 + lane;
            // the pair's Gaussian: the last lane whose first pair is at or
            // before q (pre is non-decreasing over the lanes)
            int src = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int pc = __shfl_sync(0xffffffffu, pre, src + step);
                if (pc <= q) src += step;
            }
            const uint32_t mlo = __shfl_sync(0xffffffffu, (uint32_t)mask, src);
            const uint32_t mhi = __shfl_sync(0xffffffffu, (uint32_t)(mask >> 32), src);
            const int psrc = __shfl_sync(0xffffffffu, pre, src);
            if (q >= total) continue;  // no shuffle follows in this round
            // its camera: set bit number q - psrc of the Gaussian's mask
            uint64_t mm = ((uint64_t)mhi << 32) | mlo;
            for (int j = q - psrc; j > 0; --j) mm &= mm - 1;
            const int k = __ffsll((long long)mm) - 1;
            const int64_t i = g0 + src;
            const float mu[3] = {P.g.mean[i], P.g.mean[n + i], P.g.mean[2 * n + i]};
            const float q0[4] = {P.g.quat[i], P.g.quat[n + i], P.g.quat[2 * n + i],
                                 P.g.quat[3 * n + i]};
            const float s[3] = {P.g.scale[i], P.g.scale[n + i], P.g.scale[2 * n + i]};
            const float qn = sqrtf(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
            const float iq = 1.f / qn;
            const float w = q0[0] * iq, x = q0[1] * iq, y = q0[2] * iq, z = q0[3] * iq;
            float R[3][3];
            R[0][0] = 1.f - 2.f * (y * y + z * z);
            R[0][1] = 2.f * (x * y - w * z);
            R[0][2] = 2.f * (x * z + w * y);
            R[1][0] = 2.f * (x * y + w * z);
            R[1][1] = 1.f - 2.f * (x * x + z * z);
            R[1][2] = 2.f * (y * z - w * x);
            R[2][0] = 2.f * (x * z - w * y);
            R[2][1] = 2.f * (y * z + w * x);
            R[2][2] = 1.f - 2.f * (x * x + y * y);
            const float is[3] = {1.f / s[0], 1.f / s[1], 1.f / s[2]};
            float M[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[a][b] = R[a][b] * s[b];

            float g_mu[3] = {0.f, 0.f, 0.f}, g_R[3][3] = {}, g_s[3] = {0.f, 0.f, 0.f};
            float g_th[3] = {0.f, 0.f, 0.f};  // rotation R -> R exp([theta]_x)
            float g_op = 0.f, g_k = 0.f;
            float g_sh[n_sh][3];
#pragma unroll
            for (int kk = 0; kk < n_sh; ++kk) g_sh[kk][0] = g_sh[kk][1] = g_sh[kk][2] = 0.f;
            {
                const size_t t = (size_t)k * (size_t)n + (size_t)i;
                const DevCam& cam = P.tab->cam[k];
                float gr[GREC_FLOATS];
                const double2* src = reinterpret_cast<const double2*>(P.grec + t * GREC_FLOATS);
#pragma unroll
                for (int q = 0; q < GREC_FLOATS / 2; ++q) {
                    const double2 f = src[q];
                    gr[2 * q] = (float)f.x;
                    gr[2 * q + 1] = (float)f.y;
                }
                g_op += gr[G_OP];
                g_k += gr[G_K];

                // ---- colour -> SH and viewing direction
                {
                    float d[3] = {mu[0] - cam.C[0], mu[1] - cam.C[1], mu[2] - cam.C[2]};
                    const float len = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    const float il = 1.f / len;
                    d[0] *= il; d[1] *= il; d[2] *= il;
                    float Y[16];
                    sh_eval_basis(d[0], d[1], d[2], DEG, Y);
                    float dY[16][3];
                    sh_eval_basis_grad(d[0], d[1], d[2], DEG, dY);
                    float g_dir[3] = {0.f, 0.f, 0.f};
                    const size_t shb = (size_t)i * n_sh * 3;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        float hc[n_sh];
                        float raw = 0.5f;
#pragma unroll
                        for (int kk = 0; kk < n_sh; ++kk) {
                            hc[kk] = load_feat(P.g.sh, shb + kk * 3 + ch, P.g.feat_dtype);
                            raw = fmaf(Y[kk], hc[kk], raw);
                        }
                        if (raw < 0.f) continue;  // clamped at 0
                        const float gc = gr[G_RGB + ch];
#pragma unroll
                        for (int kk = 0; kk < n_sh; ++kk) {
                            g_sh[kk][ch] = fmaf(Y[kk], gc, g_sh[kk][ch]);
                            const float h = hc[kk] * gc;
                            g_dir[0] = fmaf(h, dY[kk][0], g_dir[0]);
                            g_dir[1] = fmaf(h, dY[kk][1], g_dir[1]);
                            g_dir[2] = fmaf(h, dY[kk][2], g_dir[2]);
                        }
                    }
                    const float dd = g_dir[0] * d[0] + g_dir[1] * d[1] + g_dir[2] * d[2];
                    for (int a = 0; a < 3; ++a) g_mu[a] += (g_dir[a] - dd * d[a]) * il;
                }

                // ---- projection, EWA covariance, conic
                const float* Wr = cam.R_wc;
                const float pc[3] = {Wr[0] * mu[0] + Wr[1] * mu[1] + Wr[2] * mu[2] + cam.t_wc[0],
                                     Wr[3] * mu[0] + Wr[4] * mu[1] + Wr[5] * mu[2] + cam.t_wc[1],
                                     Wr[6] * mu[0] + Wr[7] * mu[1] + Wr[8] * mu[2] + cam.t_wc[2]};
                const float iz = 1.f / pc[2];
                const float J00 = cam.fx * iz, J11 = cam.fy * iz;
                const float J02 = -cam.fx * pc[0] * iz * iz, J12 = -cam.fy * pc[1] * iz * iz;
                float Tm[2][3];
                for (int j = 0; j < 3; ++j) {
                    Tm[0][j] = J00 * Wr[j] + J02 * Wr[6 + j];
                    Tm[1][j] = J11 * Wr[3 + j] + J12 * Wr[6 + j];
                }
                // The record holds G' = dL/d(2D covariance) in the splat's
                // principal frame E (columns e0 = (ec, es), e1 = (-es, ec)), so
                // G = E G' E^T.  With V' = E^T T M (M = R S: the projected scaled
                // axes in that frame) every product below stays free of
                // cancellation, also for a thin splat seen far off-axis, where
                // T^T G T has entries orders of magnitude above the gradients.
                const float* rp = P.rec + t * REC_FLOATS;
                const float ec = rp[R_EC], es = rp[R_ES];
                // the long-axis row in float32 here; the short-axis row, orders of
                // magnitude below T M's entries for a thin splat seen far
                // off-axis, from the preprocess's double-float chain
                float Vp[2][3];
                {
                    const float4 v1 = P.vp[t];
                    Vp[1][0] = v1.x;
                    Vp[1][1] = v1.y;
                    Vp[1][2] = v1.z;
                }
                for (int j = 0; j < 3; ++j) {
                    float tm[2];
                    for (int a = 0; a < 2; ++a)
                        tm[a] = Tm[a][0] * M[0][j] + Tm[a][1] * M[1][j] + Tm[a][2] * M[2][j];
                    Vp[0][j] = ec * tm[0] + es * tm[1];
                }
                const float Gp[2][2] = {{gr[G_CA], 0.5f * gr[G_CB]}, {0.5f * gr[G_CB], gr[G_CC]}};
                float GV[2][3];
                for (int a = 0; a < 2; ++a)
                    for (int j = 0; j < 3; ++j) GV[a][j] = Gp[a][0] * Vp[0][j] + Gp[a][1] * Vp[1][j];
                // H = V'^T G' V' = S (T R)^T G (T R) S.  Sigma = R S^2 R^T:
                // dL/ds_b = 2 H_bb / s_b, and for R -> R exp([theta]_x)
                // dL/dtheta_k = 2 (s_i / s_j - s_j / s_i) H_ij, (i, j, k) cyclic
                float H[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) H[a][b] = Vp[0][a] * GV[0][b] + Vp[1][a] * GV[1][b];
                for (int b = 0; b < 3; ++b) g_s[b] += 2.f * H[b][b] * is[b];
                g_th[0] += 2.f * (s[1] * is[2] - s[2] * is[1]) * H[1][2];
                g_th[1] += 2.f * (s[2] * is[0] - s[0] * is[2]) * H[2][0];
                g_th[2] += 2.f * (s[0] * is[1] - s[1] * is[0]) * H[0][1];
                // dL/dT = 2 G T Sigma = 2 E (G' V') M^T
                float gT[2][3];
                {
                    float EGV[2][3];
                    for (int j = 0; j < 3; ++j) {
                        EGV[0][j] = ec * GV[0][j] - es * GV[1][j];
                        EGV[1][j] = es * GV[0][j] + ec * GV[1][j];
                    }
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 3; ++b)
                            gT[a][b] = 2.f * (EGV[a][0] * M[b][0] + EGV[a][1] * M[b][1] +
                                              EGV[a][2] * M[b][2]);
                }
                const float gJ00 = gT[0][0] * Wr[0] + gT[0][1] * Wr[1] + gT[0][2] * Wr[2];
                const float gJ02 = gT[0][0] * Wr[6] + gT[0][1] * Wr[7] + gT[0][2] * Wr[8];
                const float gJ11 = gT[1][0] * Wr[3] + gT[1][1] * Wr[4] + gT[1][2] * Wr[5];
                const float gJ12 = gT[1][0] * Wr[6] + gT[1][1] * Wr[7] + gT[1][2] * Wr[8];
                float g_pc[3];
                g_pc[0] = gJ02 * (-cam.fx * iz * iz) + gr[G_MX] * cam.fx * iz;
                g_pc[1] = gJ12 * (-cam.fy * iz * iz) + gr[G_MY] * cam.fy * iz;
                g_pc[2] = -gJ00 * cam.fx * iz * iz + gJ02 * 2.f * cam.fx * pc[0] * iz * iz * iz -
                          gJ11 * cam.fy * iz * iz + gJ12 * 2.f * cam.fy * pc[1] * iz * iz * iz -
                          gr[G_MX] * cam.fx * pc[0] * iz * iz - gr[G_MY] * cam.fy * pc[1] * iz * iz +
                          gr[G_Z];
                for (int a = 0; a < 3; ++a)
                    g_mu[a] += Wr[a] * g_pc[0] + Wr[3 + a] * g_pc[1] + Wr[6 + a] * g_pc[2];

                // ---- ray-ellipsoid setup (Sec. 3.2): v_s = S^-1 R^T (C - mu) and
                // d_s = S^-1 R^T d.  The record holds g_vs and B (= g_vs (x) v_s +
                // g_ds (x) d_s, accumulated in a form free of cancellation), so
                //   dL/ds_a = -B[a][a] / s_a,
                //   dL/dtheta_k = sum_ij eps_ijk (s_j / s_i) B[i][j],
                //   dL/dmu = -R (g_vs / s).
                {
                    const float* Bm = gr + G_B;
#pragma unroll
                    for (int a = 0; a < 3; ++a) g_s[a] -= Bm[4 * a] * is[a];
                    g_th[0] += s[2] * is[1] * Bm[5] - s[1] * is[2] * Bm[7];
                    g_th[1] += s[0] * is[2] * Bm[6] - s[2] * is[0] * Bm[2];
                    g_th[2] += s[1] * is[0] * Bm[1] - s[0] * is[1] * Bm[3];
                    for (int kk = 0; kk < 3; ++kk)
                        g_mu[kk] -= R[kk][0] * gr[G_VS] * is[0] + R[kk][1] * gr[G_VS + 1] * is[1] +
                                    R[kk][2] * gr[G_VS + 2] * is[2];
                }
                // N_w[a][b] = R[a][b] / s_b
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const float gnw = gr[G_NW + 3 * a + b];
                        g_R[a][b] += gnw * is[b];
                        g_s[b] -= gnw * R[a][b] * is[b] * is[b];
                    }
            }
            // this pair's share of the Gaussian's sums
            float* row = acc + src * ACCS;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                atomicAdd(row + a, g_mu[a]);
                atomicAdd(row + 12 + a, g_s[a]);
                atomicAdd(row + 15 + a, g_th[a]);
#pragma unroll
                for (int b = 0; b < 3; ++b) atomicAdd(row + 3 + 3 * a + b, g_R[a][b]);
            }
            atomicAdd(row + 18, g_op);
            atomicAdd(row + 19, g_k);
#pragma unroll
            for (int kk = 0; kk < n_sh; ++kk)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) atomicAdd(row + 20 + 3 * kk + ch, g_sh[kk][ch]);
        }
        __syncwarp();
        if (own < n) {
            const int64_t i = own;
            const float q0[4] = {P.g.quat[i], P.g.quat[n + i], P.g.quat[2 * n + i],
                                 P.g.quat[3 * n + i]};
            const float qn = sqrtf(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
            const float iq = 1.f / qn;
            const float w = q0[0] * iq, x = q0[1] * iq, y = q0[2] * iq, z = q0[3] * iq;
            float R[3][3];
            R[0][0] = 1.f - 2.f * (y * y + z * z);
            R[0][1] = 2.f * (x * y - w * z);
            R[0][2] = 2.f * (x * z + w * y);
            R[1][0] = 2.f * (x * y + w * z);
            R[1][1] = 1.f - 2.f * (x * x + z * z);
            R[1][2] = 2.f * (y * z - w * x);
            R[2][0] = 2.f * (x * z - w * y);
            R[2][1] = 2.f * (y * z + w * x);
            R[2][2] = 1.f - 2.f * (x * x + y * y);
            const float* row = acc + lane * ACCS;
            float g_mu[3], g_R[3][3], g_s[3], g_th[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                g_mu[a] = row[a];
                g_s[a] = row[12 + a];
                g_th[a] = row[15 + a];
#pragma unroll
                for (int b = 0; b < 3; ++b) g_R[a][b] = row[3 + 3 * a + b];
            }
            const float g_op = row[18], g_k = row[19];
            float g_sh[n_sh][3];
#pragma unroll
            for (int kk = 0; kk < n_sh; ++kk)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) g_sh[kk][ch] = row[20 + 3 * kk + ch];
            // the rotation's local-frame gradient as a matrix gradient:
            // 1/2 R [g_theta]_x has the same derivative along every tangent R [e]_x
            {
                const float K[3][3] = {{0.f, -g_th[2], g_th[1]},
                                       {g_th[2], 0.f, -g_th[0]},
                                       {-g_th[1], g_th[0], 0.f}};
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        g_R[a][b] += 0.5f * (R[a][0] * K[0][b] + R[a][1] * K[1][b] + R[a][2] * K[2][b]);
            }
            // R(q^) -> q^ -> q
            const float gw = 2.f * (-z * g_R[0][1] + y * g_R[0][2] + z * g_R[1][0] - x * g_R[1][2] -
                                    y * g_R[2][0] + x * g_R[2][1]);
            const float gx = 2.f * (y * g_R[0][1] + z * g_R[0][2] + y * g_R[1][0] - 2.f * x * g_R[1][1] -
                                    w * g_R[1][2] + z * g_R[2][0] + w * g_R[2][1] - 2.f * x * g_R[2][2]);
            const float gy = 2.f * (-2.f * y * g_R[0][0] + x * g_R[0][1] + w * g_R[0][2] + x * g_R[1][0] +
                                    z * g_R[1][2] - w * g_R[2][0] + z * g_R[2][1] - 2.f * y * g_R[2][2]);
            const float gz = 2.f * (-2.f * z * g_R[0][0] - w * g_R[0][1] + x * g_R[0][2] + w * g_R[1][0] -
                                    2.f * z * g_R[1][1] + y * g_R[1][2] + x * g_R[2][0] + y * g_R[2][1]);
            const float dq = gw * w + gx * x + gy * y + gz * z;
            const float g_q[4] = {(gw - dq * w) * iq, (gx - dq * x) * iq, (gy - dq * y) * iq,
                                  (gz - dq * z) * iq};

            const unigs_param_grads& O = P.out;
            const bool acc = O.accumulate != 0;
#define PUT(ptr, j, val) \
        do { if (ptr) { if (acc) (ptr)[j] += (val); else (ptr)[j] = (val); } } while (0)
            for (int a = 0; a < 3; ++a) {
                PUT(O.mean, a * n + i, g_mu[a]);
                PUT(O.scale, a * n + i, g_s[a]);
            }
            for (int a = 0; a < 4; ++a) PUT(O.quat, a * n + i, g_q[a]);
            PUT(O.opacity, i, g_op);
            PUT(O.kfac, i, g_k);
#pragma unroll
            for (int kk = 0; kk < n_sh; ++kk)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) PUT(O.sh, ((size_t)i * n_sh + kk) * 3 + ch, g_sh[kk][ch]);
#undef PUT
        }
        // the rows are rewritten for the next 32 Gaussians only after every
        // lane has read its own
        __syncwarp();
    }
}

template <int NS, int B>
static void launch_bwd_t(const BwdParams& P, int grid, cudaStream_t st) {
    using Smem = BwdSmem<NS, B>;
    static_assert(offsetof(Smem, gO) % 256 == 0,
                  "the upstream-gradient tile must sit at a multiple of 256 bytes");
    const size_t smem = sizeof(BwdSmem<NS, B>);
    // a failure here surfaces as the launch error the entry point returns
    ensure_smem_limit(reinterpret_cast<const void*>(&render_bwd_kernel<NS, B>), (int)smem);
    render_bwd_kernel<NS, B><<<grid, 256, smem, st>>>(P);
}

template <int B>
static void launch_bwd_b(const BwdParams& P, int grid, cudaStream_t st) {
    if (P.n_sem <= 8)
        launch_bwd_t<8, B>(P, grid, st);
    else if (P.n_sem <= 16)
        launch_bwd_t<16, B>(P, grid, st);
    else if (P.n_sem <= 32)
        launch_bwd_t<32, B>(P, grid, st);
    else
        launch_bwd_t<64, B>(P, grid, st);
}

int launch_render_bwd(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                      const unigs_outputs& fwd, const unigs_grad_outputs& go,
                      const unigs_param_grads& grads, cudaStream_t st) {
    int launches = 0;
    double* grec = ws_ptr<double>(ws, p, OFF_GREC);
    if (p.n > 0) {
        // zero the records the composite may accumulate into: those of the
        // (camera, Gaussian) pairs with a kept tile
        const int64_t total = p.n * (int64_t)p.n_cams;
        const int64_t blocks = (total + 255) / 256;
        const int64_t cap = (int64_t)sm_count() * 16;
        const int grid = (int)(blocks < cap ? blocks : cap);
        grec_zero_kernel<<<grid, 256, 0, st>>>(ws_ptr<uint32_t>(ws, p, OFF_TOUCH),
                                               reinterpret_cast<double2*>(grec), total);
        ++launches;
    }
    if (grads.sem && !grads.accumulate && p.n_sem > 0)
        cudaMemsetAsync(grads.sem, 0, sizeof(float) * (size_t)p.n * p.n_sem, st);
    if (p.n_tiles > 0 && p.n > 0 && bwd_tc_selected(p)) {
        launches += launch_render_bwd_tc(p, g, ws, fwd, go, grads, grec, st);
    } else if (p.n_tiles > 0 && p.n > 0) {
        BwdParams P;
        P.tab = ws_ptr<CamTable>(ws, p, OFF_CAM);
        P.n_cams = p.n_cams;
        P.n_sem = p.n_sem;
        P.n = p.n;
        P.n_tiles = p.n_tiles;
        P.rec = ws_ptr<float>(ws, p, OFF_REC);
        // bfloat16 logits are read from their float32 copy (made by the preprocess)
        P.sem = p.feat_dtype ? ws_ptr<float>(ws, p, OFF_SEM32) : static_cast<const float*>(g.sem);
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
        P.sem_bulk = (p.n_sem > 0) && ((p.n_sem * 4) % 16 == 0) &&
                     ((reinterpret_cast<uintptr_t>(P.sem) & 15) == 0);
        cudaMemsetAsync(P.work, 0, sizeof(uint32_t), st);
        // default shape: batch 8, 3 CTAs per SM
        const int batch = p.cfg.batch > 0 ? p.cfg.batch : 8;
        const int ctas = p.cfg.ctas_per_sm > 0 ? p.cfg.ctas_per_sm : 3;
        int64_t grid = (int64_t)sm_count() * ctas;
        if (grid > p.n_tiles) grid = p.n_tiles;
        switch (batch) {
            case 8: launch_bwd_b<8>(P, (int)grid, st); break;
            case 16: launch_bwd_b<16>(P, (int)grid, st); break;
            case 64: launch_bwd_b<64>(P, (int)grid, st); break;
            default: launch_bwd_b<32>(P, (int)grid, st); break;
        }
        ++launches;
    }
    if (p.n > 0) {
        PreBwdParams Q;
        Q.tab = ws_ptr<CamTable>(ws, p, OFF_CAM);
        Q.n_cams = p.n_cams;
        Q.g = g;
        Q.rec = ws_ptr<float>(ws, p, OFF_REC);
        Q.grec = grec;
        Q.vp = ws_ptr<float4>(ws, p, OFF_VP);
        Q.touched = ws_ptr<uint32_t>(ws, p, OFF_TOUCH);
        Q.out = grads;
        Q.lowpass = p.cfg.lowpass;
        const int64_t blocks = (p.n + PREBWD_THREADS - 1) / PREBWD_THREADS;
        const int64_t cap = (int64_t)sm_count() * 32;
        const int grid = (int)(blocks < cap ? blocks : cap);
        switch (g.sh_degree) {
            case 0: preprocess_bwd_kernel<0><<<grid, PREBWD_THREADS, 0, st>>>(Q); break;
            case 1: preprocess_bwd_kernel<1><<<grid, PREBWD_THREADS, 0, st>>>(Q); break;
            case 2: preprocess_bwd_kernel<2><<<grid, PREBWD_THREADS, 0, st>>>(Q); break;
            default: preprocess_bwd_kernel<3><<<grid, PREBWD_THREADS, 0, st>>>(Q); break;
        }
        ++launches;
    }
    return launches;
}

}  // namespace unigs
