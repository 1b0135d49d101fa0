/*
 * unigs.h - C ABI of the GB300 (sm_103a) UniGS multimodal Gaussian rasterizer.
 *
 * One front-to-back compositing pass renders, per camera and pixel, the RGB
 * colour, the ray-ellipsoid midpoint depth (Sec. 3.2, Eq. midpoint; Eq.
 * depth_render), the composited per-Gaussian ellipsoid normal, the gradient
 * factor map K (Sec. 3.3, Eq. t_render) and the semantic logits (Sec. 3.4,
 * Eq. semantic_render), following Alg. 2.  A post-pass derives the paper's
 * normal map from the depth (Alg. 1).  The backward (Alg. 3, Alg. 4 and the
 * supplement's Sec. 2 chain for the depth) returns gradients to the means,
 * quaternions, scales, opacity, SH coefficients, semantic logits and the
 * gradient factor k of every Gaussian (Eq. 1 lists these parameters).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every pointer argument marked "device" is caller-owned device memory.
 *   The library never allocates or frees memory and keeps no global mutable
 *   state beyond host-side caches of device attributes (the SM count, and the
 *   shared-memory limit set per kernel and device, under a mutex); the caller
 *   allocates one workspace of unigs_workspace_bytes().
 *   The one exception is unigs_sort_pairs_static (end of this header): its
 *   scratch is a static device array of the library, shared by every call,
 *   with a process-wide cache of that array's address per device.
 * - All calls are asynchronous on the given CUDA stream, except
 *   unigs_bin_sort() with a non-NULL n_instances_out and unigs_status_poll(),
 *   which synchronise that stream.
 * - Host-detectable errors (NULL pointers, bad sizes, unsupported options)
 *   are returned immediately and nothing is launched.  Errors found on the
 *   device (instance capacity exceeded, a bounded wait that gave up) are
 *   recorded in a status word inside the workspace; unigs_status_poll()
 *   reads it.  No kernel traps or asserts.
 * - Images of several cameras are concatenated: camera k's block of a
 *   C-channel output starts at element C * pixel_offset[k] (pixel_offset in
 *   unigs_plan) and is laid out [C][H_k][W_k] (planar, row-major).
 * - Pixel (u, v) is sampled at integer coordinates; its ray direction in the
 *   camera frame is ((u - cx)/fx, (v - cy)/fy, 1) (Eq. computeRay; the
 *   supplement's back-projection uses cx = W/2, cy = H/2).  Camera frame: x
 *   right, y down, z forward.
 * - Tiles are tile_w x tile_h pixels (unigs_config; 16 x 16 by default, or
 *   8 x 32, 32 x 8, 64 x 4: always 256 pixels, one per thread of a composite
 *   CTA), numbered per camera row-major and offset by the tiles of the
 *   preceding cameras (global tile id).
 */
#ifndef UNIGS_H
#define UNIGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* unigs_stream; /* a cudaStream_t; NULL = legacy default */

#define UNIGS_MAX_CAMS 64
#define UNIGS_TILE 16         /* default tile side */
#define UNIGS_TILE_PIXELS 256 /* pixels of every tile shape */
#define UNIGS_MAX_SEM 64

typedef enum {
    UNIGS_OK = 0,
    UNIGS_ERR_INVALID_ARG = 1, /* host-side argument check failed               */
    UNIGS_ERR_CAPACITY = 2,    /* more (tile, Gaussian) instances than capacity  */
    UNIGS_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed    */
    UNIGS_ERR_NONFINITE = 4,   /* a parameter array holds a NaN or an infinity
                                  (UNIGS_FLAG_CHECK_FINITE)                       */
    UNIGS_ERR_TIMEOUT = 5      /* a bounded device wait ran out                  */
} unigs_status;

/* Pinhole camera, float32.  R_wc/t_wc map world to camera (p_c = R_wc p +
 * t_wc); R_cw and C are the camera-to-world rotation and the camera centre
 * (R_cam^world and t_cam^world of Eq. computeRay).  Matrices row-major. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R_wc[9];
    float t_wc[3];
    float R_cw[9];
    float C[3];
    float z_near; /* Gaussians with camera-frame z <= z_near are culled (0.2) */
} unigs_camera;

/* The Gaussian map G = {mu, q, s, alpha, h, o, k} of Eq. 1, device pointers.
 * mean [3][n], quat [4][n] (w,x,y,z; need not be unit), scale [3][n] (> 0),
 * opacity [n] (already activated, in (0,1)), kfac [n], sh [n][(deg+1)^2][3],
 * sem [n][n_sem].  sh and sem are float32 (feat_dtype 0) or bfloat16
 * (feat_dtype 1); every other array is float32.  All pointers 16-byte
 * aligned. */
typedef struct {
    int64_t n;
    int32_t sh_degree;  /* 0..3 */
    int32_t n_sem;      /* 0..UNIGS_MAX_SEM */
    int32_t feat_dtype; /* 0 = float32, 1 = bfloat16 */
    int32_t reserved;
    const float* mean;
    const float* quat;
    const float* scale;
    const float* opacity;
    const float* kfac;
    const void* sh;
    const void* sem;
} unigs_gaussians;

/* Per-pixel outputs (device).  Layout as in the header comment.  T_final and
 * n_contrib (1-based position in the tile list of the last Gaussian blended,
 * 0 if none) are the forward state Alg. 4 restores. */
typedef struct {
    float* rgb;          /* 3 channels      */
    float* depth;        /* 1               */
    float* normal_g;     /* 3, world frame  */
    float* kmap;         /* 1               */
    float* logits;       /* n_sem           */
    float* T_final;      /* 1               */
    uint32_t* n_contrib; /* 1               */
} unigs_outputs;

/* Upstream gradients dL/d(output), device, same layouts.  NULL means zero. */
typedef struct {
    const float* rgb;
    const float* depth; /* must already include the part from the depth normal
                           (unigs_depth_normal_bwd output) */
    const float* normal_g;
    const float* kmap;
    const float* logits;
} unigs_grad_outputs;

/* Parameter gradients (device, float32 for every array, also for bf16
 * features), laid out like the parameters.  accumulate = 0 overwrites,
 * 1 adds to the existing contents. */
typedef struct {
    float* mean;
    float* quat;
    float* scale;
    float* opacity;
    float* kfac;
    float* sh;
    float* sem;
    int32_t accumulate;
    int32_t reserved;
} unigs_param_grads;

/* Compositing and normal-from-depth settings.  unigs_config_default() fills
 * alpha_min 1/255, alpha_max 0.99, T_min 1e-4, lowpass 0.3 (the 3DGS values
 * the paper keeps, Sec. 3.4), step1 1, step2 2, lambda 0.5 (Alg. 1; the
 * paper does not print its values), and 0 (= the library's choice) for every
 * launch-shape field.  unigs_plan_init rejects settings outside
 * 0 <= alpha_min <= alpha_max < 1 (the backward divides by 1 - alpha),
 * 0 <= T_min < 1 and a finite lowpass >= 0.  The launch shape changes the speed only: the forward
 * outputs do not depend on it (the tensor-core logit blend: up to float32
 * summation order), the gradients up to float32 atomic summation order. */
typedef struct {
    float alpha_min, alpha_max, T_min, lowpass;
    int32_t step1, step2; /* 1..4 */
    float lambda;
    uint32_t flags;       /* bit 0: UNIGS_FLAG_CENTER_DEPTH (depth of the
                             Gaussian centre instead of the midpoint, the
                             ablation of Tab. 6); bit 1:
                             UNIGS_FLAG_SIMT_LOGITS (blend the logits on the
                             FP32 pipes even where the tensor-core blend
                             applies); bit 2: UNIGS_FLAG_CHECK_FINITE
                             (unigs_preprocess scans every parameter array
                             and records UNIGS_ERR_NONFINITE in the status
                             word if one holds a NaN or an infinity) */
    int32_t batch;        /* Gaussians staged per batch by the backward
                             composite: 8, 16, 32 or 64 (0 = 8) */
    int32_t ctas_per_sm;  /* persistent backward CTAs per SM, 1..8 (0 = 3) */
    int32_t batch_fwd;    /* forward composite: 16, 32 or 64; 0 = 16 on the
                             tensor-core path, 32 on the FP32 pipes */
    int32_t ctas_per_sm_fwd; /* forward composite, 1..8 (the tensor-core path
                             caps it at 4); 0 = 4 on the tensor-core path, 2
                             on the FP32 pipes */
    int32_t tile_w, tile_h; /* tile shape in pixels: 16 x 16 (0 x 0 = 16 x 16),
                             8 x 32, 32 x 8 or 64 x 4.  It sets which (tile,
                             Gaussian) pairs are listed and the schedule, not
                             the rendered result: a Gaussian is drawn on the
                             pixels of its 3-sigma square (not on whole tiles),
                             so every pixel blends the same Gaussians in the
                             same order for every shape.  n_contrib (a position
                             in the tile's list) and the float32 summation
                             order of the tensor-core logit blend and of the
                             backward's atomics do depend on it */
} unigs_config;

#define UNIGS_FLAG_CENTER_DEPTH 1u
#define UNIGS_FLAG_SIMT_LOGITS 2u
#define UNIGS_FLAG_CHECK_FINITE 4u

/* Host-side plan: sizes and workspace offsets for one (Gaussians, cameras)
 * configuration.  Filled by unigs_plan_init; owned by the caller; read-only
 * for every other call. */
typedef struct {
    int64_t n;
    int32_t n_cams, n_sem, sh_degree, feat_dtype;
    int64_t capacity;       /* instance capacity (tile, Gaussian pairs) */
    int64_t n_tiles;        /* all cameras */
    int64_t n_pixels;       /* all cameras */
    int32_t tile_offset[UNIGS_MAX_CAMS + 1];
    int64_t pixel_offset[UNIGS_MAX_CAMS + 1];
    int32_t sort_passes;    /* 8-bit radix passes over the used key bits */
    int32_t reserved;
    size_t ws_bytes;
    size_t off[20];         /* internal region offsets */
    unigs_config cfg;
} unigs_plan;

void unigs_config_default(unigs_config* cfg);

/* Validates the sizes, fills *plan and its workspace size.  instance_capacity
 * bounds the number of (tile, Gaussian) pairs over all cameras (the 3DGS
 * duplication step); 0 picks 4 * n * n_cams.  cams is host memory.  The
 * plan's cfg holds the resolved tile shape (16 x 16 for 0 x 0).
 * Returns UNIGS_ERR_INVALID_ARG on n < 0, n_cams outside 1..UNIGS_MAX_CAMS,
 * n * n_cams >= 2^32 (the device lists index (camera, Gaussian) pairs in 32
 * bits; the workspace, over 500 bytes a pair, would not fit anyway), an empty
 * image, sh_degree outside 0..3, n_sem outside 0..64, a tile shape other than
 * the four listed in unigs_config. */
unigs_status unigs_plan_init(unigs_plan* plan, const unigs_gaussians* g,
                             const unigs_camera* cams, int32_t n_cams,
                             const unigs_config* cfg, int64_t instance_capacity);

size_t unigs_workspace_bytes(const unigs_plan* plan);

/* Preprocess (per camera x Gaussian): projection, EWA 2D
 * covariance with the low-pass, 3-sigma tile rectangle, SH colour, the
 * per-Gaussian ray-ellipsoid setup of Sec. 3.2 (v_s = S^-1 R^T (C - mu) and
 * the camera-ray map S^-1 R^T R_cw) and the depth key.  The tile rectangle
 * and key follow an explicit float32 recipe (bit-reproducible).  Two passes:
 * the culling pass (one thread per pair) decides the tiles and lists the
 * pairs with a kept tile; the splat pass (one thread per listed pair) writes
 * their records.  Also clears the workspace status word.  cams: host array of
 * plan->n_cams cameras.
 * With UNIGS_FLAG_CHECK_FINITE it first scans the Gaussian arrays for NaN
 * and infinity (UNIGS_ERR_NONFINITE in the status word; the stages still run,
 * and a non-finite input then gives non-finite outputs, never a hang). */
unigs_status unigs_preprocess(const unigs_plan* plan, const unigs_gaussians* g,
                              const unigs_camera* cams, void* ws, unigs_stream stream);

/* Binning: exclusive scan of tiles touched, emission of (global tile << 32 |
 * depth bits) keys with the Gaussian index as value, stable LSD radix sort of
 * the used key bits, and per-tile [start, end) ranges.  Within a tile the
 * order is (centre depth, Gaussian index).  If n_instances_out is non-NULL the
 * stream is synchronised and the instance total written there; if the total
 * exceeds plan->capacity the call returns UNIGS_ERR_CAPACITY (nothing is
 * written out of bounds; re-plan with at least that capacity).  With NULL it
 * does not synchronise (CUDA-graph capture); an overflow then sets the status
 * word and the later stages render nothing. */
unigs_status unigs_bin_sort(const unigs_plan* plan, void* ws, int64_t* n_instances_out,
                            unigs_stream stream);

/* Forward composite, Alg. 2 (T initialised to 1; k blended, not t; colour
 * from SH; each Gaussian truncated to its 3-sigma square |u - m_x| <= r,
 * |v - m_y| <= r with r = ceil(3 sqrt(lambda_max)) of the binning recipe, the
 * 3DGS radius applied per pixel): persistent CTAs pull tiles longest list first, Gaussian
 * batches staged in shared memory by bulk (TMA) copies, per-pixel
 * accumulators in registers, early exit when every pixel of the tile has
 * T < T_min.  With 9..64 logits (and without UNIGS_FLAG_SIMT_LOGITS) the
 * logit blend of Eq. semantic_render runs on the tensor cores as a per-batch
 * product W F (weights split into two bfloat16 parts, float32 features into
 * two more, float32 accumulation in tensor memory); the other channels do
 * not change.  Non-finite logits are outside the contract (on the tensor-core
 * path they reach every pixel of the tile batch). */
unigs_status unigs_render_fwd(const unigs_plan* plan, const unigs_gaussians* g, void* ws,
                              const unigs_outputs* out, unigs_stream stream);

/* Normal from depth, Alg. 1 with the supplement's back-projection and view
 * correction: central differences of the back-projected depth at step1 and
 * step2, n2 aligned to n1 (sign(0) = +1), lambda fusion, normalisation,
 * flipped to face the camera.  normal_d: 3 channels, world frame; 0 where a
 * stencil point falls outside the image or the fused vector is 0.  depth and
 * normal_d are device arrays in the concatenated layout. */
unigs_status unigs_depth_normal_fwd(const unigs_plan* plan, const unigs_camera* cams,
                                    const float* depth, float* normal_d, unigs_stream stream);

/* Alg. 3: dL/dDepth from dL/dNormal_d, written as a deterministic gather
 * (each pixel sums the terms of the stencils that contain it; the paper
 * scatters with atomics).  g_depth_out = g_depth_in + dL/dDepth; g_depth_in
 * may be NULL (zero) or equal g_depth_out. */
unigs_status unigs_depth_normal_bwd(const unigs_plan* plan, const unigs_camera* cams,
                                    const float* depth, const float* g_normal_d,
                                    const float* g_depth_in, float* g_depth_out,
                                    unigs_stream stream);

/* Backward composite, Alg. 4 (reverse order from n_contrib, T <- T/(1-alpha),
 * per-channel weights w = alpha T), with warp-level pre-reduction before
 * float32 atomics into per-(camera, Gaussian) intermediate gradients, then
 * the per-Gaussian chain to mu, q (tangent projection of the normalised
 * quaternion), s, opacity, SH, k and the logits (supplement Sec. 2 for the
 * depth; the EWA and SH chain of 3DGS for the rest).  fwd must hold the
 * T_final / n_contrib of the matching unigs_render_fwd.  Each call first
 * zeroes the per-(camera, Gaussian) gradient records it accumulates into
 * (the pairs with a kept tile), so several backward passes may follow one
 * forward. */
unigs_status unigs_render_bwd(const unigs_plan* plan, const unigs_gaussians* g,
                              const unigs_camera* cams, void* ws, const unigs_outputs* fwd,
                              const unigs_grad_outputs* grad_out, unigs_param_grads* grads,
                              unigs_stream stream);

/* Reads the workspace status word (synchronises the stream).  *detail gets
 * the required instance count for UNIGS_ERR_CAPACITY, and for
 * UNIGS_ERR_NONFINITE the first array found non-finite (0 mean, 1 quat,
 * 2 scale, 3 opacity, 4 kfac, 5 sh, 6 sem).  Device-side values:
 * UNIGS_ERR_CAPACITY, UNIGS_ERR_NONFINITE, UNIGS_ERR_TIMEOUT, and
 * UNIGS_ERR_CUDA when the
 * backward composite finds its dynamic shared memory not aligned to its
 * 256-byte row layout (the kernel then does no work). */
unigs_status unigs_status_poll(const unigs_plan* plan, const void* ws, int64_t* detail,
                               unigs_stream stream);

/* Work counters of the last unigs_render_fwd on this workspace (synchronises
 * the stream): the (pixel, Gaussian) pairs whose alpha was evaluated, and the
 * pairs blended (alpha >= alpha_min before the transmittance stop).  These
 * are the units of the compositing cost model.  Cleared by unigs_preprocess. */
unigs_status unigs_stats_poll(const unigs_plan* plan, const void* ws, int64_t* pairs_evaluated,
                              int64_t* pairs_blended, unigs_stream stream);

/* The number of kernels one preprocess + bin_sort + render_fwd +
 * depth_normal_fwd + depth_normal_bwd + render_bwd sequence launches for this
 * plan (the count is fixed by the plan). */
int32_t unigs_launches_per_step(const unigs_plan* plan);

/* The composite kernels this plan runs, fixed at plan time by the logit width,
 * the feature dtype, UNIGS_FLAG_SIMT_LOGITS and the launch shapes: a bit set
 * of UNIGS_PATH_*.  UNIGS_PATH_FWD_TC: the forward blends the logits on the
 * tensor cores (9..64 logits).  UNIGS_PATH_BWD_TC: the backward forms the
 * logit terms of Alg. 4 on the tensor cores (bfloat16 logits, 9..64 of them,
 * backward shape default or batch 16 x 2 CTAs per SM).  UNIGS_PATH_SEM32:
 * unigs_preprocess makes a float32 copy of bfloat16 logit rows for an
 * FP32-pipe composite.  0 for a NULL plan. */
#define UNIGS_PATH_FWD_TC 1
#define UNIGS_PATH_BWD_TC 2
#define UNIGS_PATH_SEM32 4
int32_t unigs_plan_paths(const unigs_plan* plan);

const char* unigs_status_string(unigs_status s);

/* Allocation-free sort (the paper has no counterpart: this is a service for
 * callers that cannot allocate device memory where they call, e.g. code with a
 * memory budget fixed at start-up, a plugin host that owns every allocation,
 * or a real-time loop in which a cudaMalloc may not run).
 *
 * Stable LSD radix sort of n (key, value) pairs by the low key_bits bits of
 * the key - the sort unigs_bin_sort runs on the tile|depth keys - but with its
 * scratch memory (one ping-pong buffer, digit histograms, scan partials, a
 * status block) in a static device array of the library rather than in a
 * caller workspace.  The caller passes device inputs and outputs only.
 * Sorted order: ascending (key mod 2^key_bits), ties in input order; key
 * bits at and above key_bits may hold anything and never decide the order
 * (the last 8-bit pass is masked to the bits that remain), and the output
 * keys are the input keys unchanged.
 *
 * Limits and behaviour: n <= UNIGS_STATIC_SORT_MAX_PAIRS (2^20); larger n,
 * key_bits outside 1..64, NULL buffers, or an output that shares a byte with
 * an input or with the other output return UNIGS_ERR_INVALID_ARG before
 * anything runs.  The static array (about
 * 12.5 MB) is held by every GPU that loads the library until the process
 * exits.  The first call on a device (with that device current, and the
 * stream on that device) looks up the array's device address; make that
 * first call before any stream capture.  Every call shares the one array and
 * overwrites it: calls that overlap on the GPU (other streams, other host
 * threads) race.  Asynchronous on the stream; calls no allocator. */
#define UNIGS_STATIC_SORT_MAX_PAIRS (1 << 20)
unigs_status unigs_sort_pairs_static(const unsigned long long* keys_in, const uint32_t* vals_in,
                                     int64_t n, int32_t key_bits, unsigned long long* keys_out,
                                     uint32_t* vals_out, unigs_stream stream);

/* FP32 FMA throughput probe (a measurement utility; the paper has no
 * counterpart).  The composite kernels are bound by FP32 arithmetic, so their
 * roofline is taken against the FMA rate measured on the GPU in use.  Launches
 * one kernel of 8 CTAs x 256 threads per SM, each thread running 8 independent
 * FMA chains of 16 * iters steps, as scalar FMAs (packed = 0) or as packed
 * float32-pair FMAs (packed = 1, two FMAs per instruction).  sink: device
 * buffer of at least unigs_probe_fma_sink_floats() floats (caller-owned,
 * receives one value per thread).  *flops_out (host, may be NULL) gets the
 * floating-point operations of the launch (an FMA counts 2).  The caller
 * times the launch on its stream.  Returns UNIGS_ERR_INVALID_ARG for a NULL
 * sink, iters < 1 or packed outside 0..1, UNIGS_ERR_CUDA if the launch fails. */
int64_t unigs_probe_fma_sink_floats(void);
unigs_status unigs_probe_fma(float* sink, int32_t iters, int32_t packed, int64_t* flops_out,
                             unigs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* UNIGS_H */
