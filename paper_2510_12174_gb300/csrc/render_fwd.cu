// Forward composite (Alg. 2): 256 threads per 16x16 tile, one pixel per
// thread, persistent CTAs.
//
// Per pixel and per Gaussian of the tile's front-to-back list: alpha from the
// 2D splat, skip below alpha_min, stop before the Gaussian that would bring T
// below T_min; w = alpha T; accumulate RGB, the ray-ellipsoid midpoint depth
// (Eq. midpoint, Eq. depth_render), the ellipsoid normal, k (Eq. t_render)
// and the logits (Eq. semantic_render) in registers; save T_final and the
// 1-based list position of the last blended Gaussian for the backward.
//
// Scheduling: a fixed grid of CTAs pulls global tile ids from a device work
// counter in the order of a tile list sorted by descending list length (all
// cameras of the plan in one launch), so long tiles start first and the tail
// is short.
//
// Staging: the list is walked in batches of B Gaussians.  Warp 0 issues one
// bulk copy (TMA engine) per Gaussian record (160 B) and per semantic row
// into a double-buffered shared-memory area completing on an mbarrier, so
// batch b+1 streams in while batch b is composited.  A warp whose 8x4 pixel
// block lies outside a Gaussian's alpha box, or whose pixels are all
// finished, skips it; the CTA moves on when all 256 pixels are finished.
#include "launch.h"
#include "splat.cuh"

namespace unigs {

constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct FwdParams {
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
    unigs_outputs out;
    float alpha_min, alpha_max, T_min;
    int center_depth;
    int sem_bulk;  // semantic rows are 16-byte multiples and aligned
};

template <int NS, int B>
struct FwdSmem {
    float rec[2][B][REC_FLOATS];
    float sem[2][B][NS];
    uint64_t bar[2];
    int tile;
    uint32_t issued[2];  // staging phases started per buffer (one thread counts)
};

template <int NS, int B>
__device__ __forceinline__ void issue_batch(const FwdParams& P, FwdSmem<NS, B>& S, int buf,
                                            uint32_t first, int count, int cam) {
    // executed by warp 0 only
    const int lane = threadIdx.x & 31;
    const uint32_t row_bytes = (uint32_t)(P.n_sem * sizeof(float));
    const uint32_t per = REC_FLOATS * 4 + (P.sem_bulk ? row_bytes : 0u);
    if (lane == 0) mbar_arrive_expect_tx(&S.bar[buf], per * (uint32_t)count);
    __syncwarp();
    for (int i = lane; i < count; i += 32) {
        const uint32_t g = P.vals[first + i];
        const size_t r = (size_t)cam * (size_t)P.n + g;
        bulk_g2s(&S.rec[buf][i][0], P.rec + r * REC_FLOATS, REC_FLOATS * 4, &S.bar[buf]);
        if (P.n_sem > 0) {
            const float* src = P.sem + (size_t)g * P.n_sem;
            if (P.sem_bulk) {
                bulk_g2s(&S.sem[buf][i][0], src, row_bytes, &S.bar[buf]);
            } else {
                for (int c = 0; c < P.n_sem; ++c) S.sem[buf][i][c] = src[c];
            }
        }
    }
}

// co[c] += w * row[c] with 16-byte shared-memory loads.
template <int NS>
__device__ __forceinline__ void accumulate_row(const float* row, float w, float (&co)[NS]) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int c = 0; c < NS / 4; ++c) {
        const float4 x = r4[c];
        co[4 * c + 0] = fmaf(w, x.x, co[4 * c + 0]);
        co[4 * c + 1] = fmaf(w, x.y, co[4 * c + 1]);
        co[4 * c + 2] = fmaf(w, x.z, co[4 * c + 2]);
        co[4 * c + 3] = fmaf(w, x.w, co[4 * c + 3]);
    }
}

template <int NS, int B>
__global__ void __launch_bounds__(256, 2) render_fwd_kernel(const FwdParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FwdSmem<NS, B>& S = *reinterpret_cast<FwdSmem<NS, B>*>(smem_raw);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    // once per CTA: zero the semantic padding (rows shorter than NS), init barriers
    for (int j = tid; j < 2 * B * NS; j += 256) (&S.sem[0][0][0])[j] = 0.f;
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
        S.issued[0] = S.issued[1] = 0u;
    }
    __syncthreads();
    // phases waited for per buffer (uniform across the CTA): the parity of the
    // next phase to wait for
    uint32_t loads0 = 0u, loads1 = 0u;
    bool timed_out = false;
    // Warp 0 stages a batch unless one of its own waits gave up (a
    // warp-uniform decision: lane 0 arms the barrier, every lane issues
    // copies).  Warp 0 waits on every phase itself, so a buffer is restaged
    // only after its previous copy was seen to land: at most one copy per
    // buffer is ever in flight, and the exit drain finds it by S.issued.
    auto issue = [&](int bf, uint32_t first, int cnt, int cam) {
        if (__any_sync(0xffffffffu, timed_out)) return;
        issue_batch<NS, B>(P, S, bf, first, cnt, cam);
        if ((tid & 31) == 0) ++S.issued[bf];
    };
    // every thread waits for the batch in buffer bf (bounded)
    auto wait_batch = [&](int bf) {
        const uint32_t ph = bf ? loads1 : loads0;
        if (!mbar_wait_bounded(&S.bar[bf], ph & 1u, WAIT_LIMIT)) timed_out = true;
        if (bf) ++loads1; else ++loads0;
    };
    uint32_t n_eval = 0, n_blend = 0;

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
        if (warp == 0 && n_batches > 0) issue(0, range.x, min(B, n_items), cam_idx);
        // rows staged with plain stores (unaligned semantic rows) must be
        // visible before the first batch is read; later batches are ordered by
        // the end-of-batch barrier
        __syncthreads();

        float T = 1.f;
        float crgb[3] = {0.f, 0.f, 0.f}, cdep = 0.f, cn[3] = {0.f, 0.f, 0.f}, ck = 0.f;
        float co[NS];
#pragma unroll
        for (int c = 0; c < NS; ++c) co[c] = 0.f;
        uint32_t last = 0;
        bool done = !inside;

        for (int b = 0; b < n_batches; ++b) {
            const int buf = b & 1;
            if (warp == 0 && b + 1 < n_batches)
                issue(buf ^ 1, range.x + (b + 1) * B, min(B, n_items - (b + 1) * B), cam_idx);
            wait_batch(buf);
            const int count = min(B, n_items - b * B);
            const bool skip = __all_sync(0xffffffffu, done || timed_out);
            if (!skip) {
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
                    accumulate_row<NS>(&S.sem[buf][j][0], w, co);
                    T = test_T;
                    last = (uint32_t)(b * B + j + 1);
                }
            }
            const int alive = __syncthreads_count(!done && !timed_out);
            if (alive == 0) {
                // drain the batch already in flight before leaving the tile
                if (b + 1 < n_batches) wait_batch(buf ^ 1);
                break;
            }
        }
        if (inside) {
            const int W = cam.width;
            const int64_t HW = (int64_t)cam.height * W;
            const int64_t pix = cam.pix_off;
            const int64_t idx = (int64_t)v * W + u;
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
            if (P.out.logits) {
                float* lo = P.out.logits + pix * (int64_t)P.n_sem + idx;
#pragma unroll
                for (int c = 0; c < NS; ++c)
                    if (c < P.n_sem) lo[(int64_t)c * HW] = co[c];
            }
        }
        // the end-of-batch barrier already separated this tile's last use of
        // the shared buffers from the next tile's first issue; a bounded wait
        // that gave up ends the CTA (uniformly)
        if (__syncthreads_or(timed_out)) break;
    }
    // no bulk copy may still be landing in this CTA's shared memory when it
    // exits (after a timeout the issuer stopped, so at most one per buffer)
    if (tid == 0 && !drain_bulk(S.bar, S.issued[0], S.issued[1], WAIT_LIMIT)) timed_out = true;
    if (timed_out && (tid & 31) == 0) set_status(P.hdr, UNIGS_ERR_TIMEOUT);
    // work counters: one atomic per warp
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

template <int NS, int B>
static void launch_fwd_t(const FwdParams& P, int grid, cudaStream_t st) {
    const size_t smem = sizeof(FwdSmem<NS, B>);
    // a failure here surfaces as the launch error the entry point returns
    ensure_smem_limit(reinterpret_cast<const void*>(&render_fwd_kernel<NS, B>), (int)smem);
    render_fwd_kernel<NS, B><<<grid, 256, smem, st>>>(P);
}

template <int B>
static void launch_fwd_b(const FwdParams& P, int grid, cudaStream_t st) {
    if (P.n_sem <= 8)
        launch_fwd_t<8, B>(P, grid, st);
    else if (P.n_sem <= 16)
        launch_fwd_t<16, B>(P, grid, st);
    else if (P.n_sem <= 32)
        launch_fwd_t<32, B>(P, grid, st);
    else
        launch_fwd_t<64, B>(P, grid, st);
}

int launch_render_fwd(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                      const unigs_outputs& out, cudaStream_t st) {
    if (p.n_tiles == 0) return 0;
    if (fwd_tc_eligible(p, g)) return launch_render_fwd_tc(p, g, ws, out, st);
    FwdParams P;
    P.tab = ws_ptr<CamTable>(ws, p, OFF_CAM);
    P.n_cams = p.n_cams;
    P.n_sem = p.n_sem;
    P.n = p.n;
    P.n_tiles = p.n_tiles;
    P.rec = ws_ptr<float>(ws, p, OFF_REC);
    // bfloat16 logits are read from their float32 copy (made by the preprocess)
    P.sem = p.feat_dtype ? ws_ptr<float>(ws, p, OFF_SEM32) : static_cast<const float*>(g.sem);
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
    P.sem_bulk = (p.n_sem > 0) && ((p.n_sem * 4) % 16 == 0) &&
                 ((reinterpret_cast<uintptr_t>(P.sem) & 15) == 0);
    cudaMemsetAsync(P.work, 0, sizeof(uint32_t), st);
    // forward shape fields, else batch 32 x 2 CTAs per SM
    const int ctas = p.cfg.ctas_per_sm_fwd > 0 ? p.cfg.ctas_per_sm_fwd : 2;
    const int batch = p.cfg.batch_fwd > 0 ? p.cfg.batch_fwd : 32;
    int64_t grid = (int64_t)sm_count() * ctas;
    if (grid > p.n_tiles) grid = p.n_tiles;
    switch (batch) {
        case 16: launch_fwd_b<16>(P, (int)grid, st); break;
        case 64: launch_fwd_b<64>(P, (int)grid, st); break;
        default: launch_fwd_b<32>(P, (int)grid, st); break;
    }
    return 1;
}

}  // namespace unigs
