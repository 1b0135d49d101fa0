// Internal definitions shared by the sm_103a kernels of libunigs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "unigs.h"

namespace unigs {

constexpr int TILE = UNIGS_TILE;             // default tile side
constexpr int TILE_PIX = UNIGS_TILE_PIXELS;  // pixels of every tile shape

// ----------------------------------------------------------------------------
// Per-(camera, Gaussian) forward record written by the preprocess and staged
// into shared memory by the composite kernels (52 floats = 208 bytes, a
// multiple of 16 so a bulk copy can move it).  The fields every evaluated
// (pixel, Gaussian) pair reads (warp box test and alpha) fill the first three
// 16-byte words.
//   [0..3]  projected centre split as integer part + remainder (x_hi, y_hi,
//           x_lo, y_lo); m = hi + lo, hi an integer-valued float, |lo| <= 0.5
//   [4..6]  conic (A, B, C) of the inverse 2D covariance; for an
//           ill-conditioned splat (flag [10]) instead the conditional form
//           q = P (a + rho b)^2 + e b^2: (P, rho_hi, rho_lo)
//   [7]     opacity
//   [8..9]  half-extents (x, y) of the box holding every pixel where alpha
//           can reach alpha_min (with margin): a warp whose 8x4 pixel block
//           lies outside skips the Gaussian
//   [10]    1 when the splat is ill-conditioned (alpha evaluated in
//           double-float), else 0
//   [11]    -1 when the camera is inside the 1-sigma ellipsoid (|v_s| <= 1),
//           else +1
//   [12..20] M_c = S^-1 R^T R_cw (camera ray -> local scaled), row-major
//   [21..23] v_s = S^-1 R^T (C - mu)
//   [24..32] N_w = R S^-1 (scaled-local normal -> world), row-major
//   [33]    camera-frame z of the centre
//   [34..36] ill-conditioned splat: e, pivot (1: a = x, b = y; 0: a = y,
//           b = x), 0; else 0
//   [37]    k (gradient factor)
//   [38..40] RGB
//   [41..43] P1, [44..46] P2: v_s x d_s = dx P1 + dy P2 for the pixel offset
//           (dx, dy) from the projected centre (see pair_geometry), the
//           cancellation-free form of the cross product for Gaussians far
//           from the camera
//   [47]    3-sigma radius r of the binning recipe (pixels): the Gaussian is
//           drawn only where |dx| <= r and |dy| <= r
//   [48..49] (cos theta, sin theta): the principal axes e0 = (cos, sin),
//           e1 = (-sin, cos) of the 2D covariance, the frame in which the
//           backward records the covariance gradient
//   [50..51] half-extents along e0 and e1 of the ellipse holding every pixel
//           where alpha can reach alpha_min (with margin): with [8..9] the
//           two boxes of the warp-block skip test
// ----------------------------------------------------------------------------
enum {
    R_MXH = 0, R_MYH, R_MXL, R_MYL, R_CON = 4, R_OP = 7, R_EXTX = 8, R_EXTY = 9,
    R_FLAG = 10, R_SR = 11, R_MC = 12, R_VS = 21, R_NW = 24, R_Z = 33, R_CLO = 34,
    R_K = 37, R_RGB = 38, R_P1 = 41, R_P2 = 44, R_R3 = 47, R_EC = 48, R_ES = 49,
    R_E0 = 50, R_E1 = 51, REC_FLOATS = 52
};

// Pixel of thread tid inside its tile of width tw (8, 16, 32 or 64; 256
// pixels): the tile is a grid of 8x4 warp blocks, tw / 8 per row; warp w
// covers the block at ((w % (tw/8)) * 8, (w / (tw/8)) * 4), lanes row-major
// within the block.
__device__ __forceinline__ void tile_pixel(int tid, int tw, int* lx, int* ly) {
    const int w = tid >> 5, lane = tid & 31, wpr = tw >> 3;
    *lx = (w % wpr) * 8 + (lane & 7);
    *ly = (w / wpr) * 4 + (lane >> 3);
}

// Origin of warp w's 8x4 block inside a tile of width tw.
__device__ __forceinline__ void warp_block(int w, int tw, int* bx, int* by) {
    const int wpr = tw >> 3;
    *bx = (w % wpr) * 8;
    *by = (w / wpr) * 4;
}

// True when the Gaussian cannot reach alpha_min anywhere in the warp's block
// [bx0, bx0+7] x [by0, by0+3] (uniform across the warp): the block lies
// outside the axis-aligned box of the q <= qlim ellipse, or outside the box
// along the ellipse's principal axes (separating-axis test of the block's
// half-extents 3.5 x 1.5 projected on e0, e1), which for an elongated splat
// is far smaller.
__device__ __forceinline__ bool warp_block_misses(const float* __restrict__ rc, float bx0,
                                                  float by0) {
    const float mx = rc[R_MXH] + rc[R_MXL], my = rc[R_MYH] + rc[R_MYL];
    const float ex = rc[R_EXTX], ey = rc[R_EXTY];
    if ((bx0 + 7.f < mx - ex) || (bx0 > mx + ex) || (by0 + 3.f < my - ey) || (by0 > my + ey))
        return true;
    const float cx = bx0 + 3.5f - mx, cy = by0 + 1.5f - my;
    const float c = rc[R_EC], s = rc[R_ES];
    const float ac = fabsf(c), as = fabsf(s);
    return fabsf(fmaf(c, cx, s * cy)) > rc[R_E0] + fmaf(3.5f, ac, 1.5f * as) ||
           fabsf(fmaf(-s, cx, c * cy)) > rc[R_E1] + fmaf(3.5f, as, 1.5f * ac);
}

// Conic eigenvalue ratio above which alpha is evaluated in double-float: the
// float32 quadratic form loses about log2(ratio) bits along the long axis.
constexpr float KAPPA_FF = 64.f;

// Per-(camera, Gaussian) intermediate gradient record (32 float64
// accumulators, 256 bytes), filled by atomics in the backward composite and
// consumed by the preprocess backward:
// dL/d(projected centre x, y), dL/d(a', b', c') of the 2D covariance
// E^T [[a, b], [b, c]] E = [[a', b'], [b', c']] in the splat's principal frame
// E (low-pass included; see the record's [48..49]), opacity, RGB, the local-frame matrix
// B = sum g_vs (x) v_s + g_ds (x) d_s (row-major, accumulated as
// g_vs (x) w + (g_ds - t g_vs) (x) d_s, see the backward composite), v_s, N_w,
// k and the centre depth (centre-depth mode).
enum {
    G_MX = 0, G_MY, G_CA, G_CB, G_CC, G_OP, G_RGB, G_B = 9, G_VS = 18,
    G_NW = 21, G_K = 30, G_Z = 31, GREC_FLOATS = 32
};

// Camera as the kernels see it (read from the workspace).
struct DevCam {
    int32_t width, height, tiles_x, tiles_y;
    int64_t tile_off, pix_off;
    float fx, fy, cx, cy;
    float R_wc[9];
    float t_wc[3];
    float R_cw[9];
    float C[3];
    float z_near;
    int32_t tile_w, tile_h;  // tile shape of the plan (the same for every camera)
    float pad;
};
static_assert(sizeof(DevCam) == 160, "DevCam layout");

struct CamTable {
    DevCam cam[UNIGS_MAX_CAMS];
};

// Device status block at the start of the workspace.
struct WsHeader {
    uint32_t status;       // unigs_status of the first device-side error
    uint32_t n_instances;  // instances emitted (valid when not overflowed)
    unsigned long long need;  // instances required (capacity errors)
    unsigned long long n_eval;   // (pixel, Gaussian) pairs whose alpha the forward evaluated
    unsigned long long n_blend;  // pairs the forward blended (alpha >= alpha_min, not stopped)
    uint32_t work_fwd;           // tile counters of the persistent composite kernels
    uint32_t work_bwd;
    uint32_t nonfinite;          // first parameter array found non-finite (flag set)
    uint32_t n_kept;             // (camera, Gaussian) pairs with a kept tile (preprocess)
    uint32_t pad[52];
};
static_assert(sizeof(WsHeader) == 256, "WsHeader layout");

// Region indices into unigs_plan::off[].
enum {
    OFF_HDR = 0, OFF_CAM, OFF_REC, OFF_RECT, OFF_TOUCH, OFF_OFFS, OFF_ZBITS,
    OFF_SCAN, OFF_KEYS0, OFF_KEYS1, OFF_VALS0, OFF_VALS1, OFF_HIST, OFF_RANGES,
    OFF_GREC, OFF_CULL, OFF_SEM32, OFF_ORDER, OFF_LOSS, OFF_VP, OFF_END
};
static_assert(OFF_END <= 20, "unigs_plan::off holds 20 region offsets");

// Per-(camera, Gaussian) record of the opacity-aware tile test (8 floats):
// float32 projected centre, float32 conic (kA, kB, kC), qlim, no-cull flag.
enum { C_MX = 0, C_MY, C_KA, C_KB, C_KC, C_QLIM, C_NOCULL, CULL_FLOATS = 8 };

// Opacity-aware tile test, float32 recipe with non-contractible operations
// (identical operation order in the oracle's binning): keep the tile when the
// minimum over its pixel-centre square of q(D) = D^T K D is <= qlim.
__device__ __forceinline__ float cull_q(float kA, float kB, float kC, float dx, float dy) {
    return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(kA, dx), dx),
                               __fmul_rn(__fmul_rn(__fmul_rn(2.f, kB), dx), dy)),
                     __fmul_rn(__fmul_rn(kC, dy), dy));
}

__device__ __forceinline__ bool tile_keep(const float* __restrict__ cr, int tx, int ty, int tw,
                                          int th) {
    if (cr[C_NOCULL] != 0.f) return true;
    const float mx = cr[C_MX], my = cr[C_MY], kA = cr[C_KA], kB = cr[C_KB], kC = cr[C_KC];
    const float X0 = (float)(tx * tw), X1 = (float)(tx * tw + tw - 1);
    const float Y0 = (float)(ty * th), Y1 = (float)(ty * th + th - 1);
    float qmin;
    if (X0 <= mx && mx <= X1 && Y0 <= my && my <= Y1) {
        qmin = 0.f;
    } else {
        const float ylo = __fsub_rn(Y0, my), yhi = __fsub_rn(Y1, my);
        const float xlo = __fsub_rn(X0, mx), xhi = __fsub_rn(X1, mx);
        float q[4];
        {
            const float dx = xlo;
            const float dy = fminf(fmaxf(__fdiv_rn(-__fmul_rn(kB, dx), kC), ylo), yhi);
            q[0] = cull_q(kA, kB, kC, dx, dy);
        }
        {
            const float dx = xhi;
            const float dy = fminf(fmaxf(__fdiv_rn(-__fmul_rn(kB, dx), kC), ylo), yhi);
            q[1] = cull_q(kA, kB, kC, dx, dy);
        }
        {
            const float dy = ylo;
            const float dx = fminf(fmaxf(__fdiv_rn(-__fmul_rn(kB, dy), kA), xlo), xhi);
            q[2] = cull_q(kA, kB, kC, dx, dy);
        }
        {
            const float dy = yhi;
            const float dx = fminf(fmaxf(__fdiv_rn(-__fmul_rn(kB, dy), kA), xlo), xhi);
            q[3] = cull_q(kA, kB, kC, dx, dy);
        }
        qmin = fminf(fminf(q[0], q[1]), fminf(q[2], q[3]));
    }
    return qmin <= cr[C_QLIM];
}

constexpr int SORT_ITEMS = 2048;   // keys per sort block (256 threads x 8)
// Tile rectangles with more tiles than this are culled-tested and emitted by
// the whole warp (32 tiles per step) rather than by their own thread: a lane
// with a long serial loop would hold its warp (measured: 4 beats 8, 16, 32).
constexpr int COOP_TILES = 4;
constexpr int SCAN_ITEMS = 4096;   // elements per scan block (256 threads x 16)
constexpr int LOSS_MAX_BLOCKS = 2048;  // block partials of the loss reduction

template <typename T>
__host__ __device__ inline T* ws_ptr(void* ws, const unigs_plan& p, int region) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + p.off[region]);
}

__device__ inline const DevCam& cam_of_tile(const CamTable* tab, int n_cams, int64_t gtile,
                                            int* cam_index) {
    int lo = 0;
    for (int k = 1; k < n_cams; ++k)
        if (gtile >= tab->cam[k].tile_off) lo = k;
    *cam_index = lo;
    return tab->cam[lo];
}

__device__ inline void set_status(WsHeader* h, uint32_t code) {
    atomicCAS(&h->status, 0u, code);
}

// Feature loads (float32 or bfloat16 storage, float32 math).
__device__ __forceinline__ float load_feat(const void* base, size_t i, int bf16) {
    if (bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[i]);
    return reinterpret_cast<const float*>(base)[i];
}

// ----------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA engine, non-tensor) helpers, inline PTX.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Adds to the expected transaction bytes of the current phase (no arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One arrival (release semantics: this thread's earlier writes are visible to
// a thread whose wait observes the phase).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Returns true once the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after max_iter polls and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t max_iter) {
    for (uint32_t i = 0; i < max_iter; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Before a CTA exits: waits (bounded) until the last bulk copy issued into
// each of the two staging buffers has landed in shared memory.  issued0/1
// count the phases started on bar[0]/bar[1]; phases complete in order and the
// producers keep at most one in flight per buffer, so the parity of the last
// one identifies it.  In a launch without timeouts every phase has already
// been waited for and this returns at once.  Returns false if a copy is still
// in flight after the limit (the caller has already recorded the timeout).
__device__ __forceinline__ bool drain_bulk(uint64_t* bar, uint32_t issued0, uint32_t issued1,
                                           uint32_t limit) {
    bool ok = true;
    if (issued0 > 0) ok &= mbar_wait_bounded(&bar[0], (issued0 - 1) & 1u, limit);
    if (issued1 > 0) ok &= mbar_wait_bounded(&bar[1], (issued1 - 1) & 1u, limit);
    return ok;
}

// 1D bulk copy global -> shared, completion counted on the mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ----------------------------------------------------------------------------
// Warp transpose-reduction: every lane holds v[32]; afterwards lane L holds
// the warp-wide sum of element L (recursive halving, 31 shuffles).  The adds
// of neighbouring elements are issued as packed float32 pairs; each element
// still sees the same additions in the same order.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float warp_reduce_transpose32(float (&v)[32], int lane) {
#pragma unroll
    for (int step = 0; step < 4; ++step) {
        const int off = 16 >> step;
        const int half = 16 >> step;  // current length is 2*half
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < half; k += 2) {
            const float2 lo = make_float2(v[k], v[k + 1]);
            const float2 hi = make_float2(v[k + half], v[k + half + 1]);
            const float2 send = upper ? lo : hi;
            const float2 keep = upper ? hi : lo;
            const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, off),
                                            __shfl_xor_sync(0xffffffffu, send.y, off));
            const float2 sum = __fadd2_rn(keep, recv);
            v[k] = sum.x;
            v[k + 1] = sum.y;
        }
    }
    const bool upper = (lane & 1) != 0;
    const float send = upper ? v[0] : v[1];
    const float keep = upper ? v[1] : v[0];
    return keep + __shfl_xor_sync(0xffffffffu, send, 1);
}

}  // namespace unigs
