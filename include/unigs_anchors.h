/*
 * unigs_anchors.h - C ABI of the anchor attribute prediction (sm_103a).
 *
 * Sec. 3.1 ("Architecture Overview", "Attribute Prediction") and Fig. 2 (a):
 * the scene is a set of anchors on a modified Scaffold-GS; every training
 * iteration, small MLPs predict from each anchor's feature the attributes
 * of its M Gaussians, which the rasterizer of unigs.h then renders.  With
 * MLP(f) = W2 relu(W1 f + b1) + b2 (two layers) and sigma the logistic
 * function, anchor a (position x, scale l > 0, offsets O_m in units of l,
 * feature f, base logits o_ah, base gradient factor k_ah) yields for
 * m = 0..M-1 the Gaussian g = a M + m:
 *   semantic logits  o_g = o_ah (x) sigma(MLP_sem(f))      (the paper's
 *                    Repeat(o_ah, M) (x) sigma(MLP_o(f_ah)); MLP_sem: R^F ->
 *                    R^n_sem, the same for every m)
 *   gradient factor  k_g = k_ah sigma(MLP_k(f))             (MLP_k: R^F -> R)
 *   opacity          alpha_g = sigma(MLP_opacity(f)_m)      (R^F -> R^M)
 *   colour           c_g = sigma(MLP_color(f)_{3m..3m+2})   (R^F -> R^3M),
 *                    stored as the degree-0 SH coefficient (c_g - 1/2) / Y_00
 *                    (Y_00 = 1 / (2 sqrt(pi))), so that the rasterizer's
 *                    colour Y_00 h + 1/2 is c_g
 *   scale            s_g = l (x) sigma(MLP_cov(f)_{7m..7m+2})   (R^F -> R^7M)
 *   rotation         q_g = MLP_cov(f)_{7m+3..7m+6} (unnormalised; the
 *                    rasterizer normalises)
 *   position         mu_g = x + l (x) O_m
 * The MLPs take the anchor feature alone (no viewing direction), as the
 * paper's MLP_o and MLP_k do.  Conventions (device pointers, streams, status
 * codes) are those of unigs.h.
 */
#ifndef UNIGS_ANCHORS_H
#define UNIGS_ANCHORS_H

#include "unigs.h"

#ifdef __cplusplus
extern "C" {
#endif

#define UNIGS_ANCHOR_FEAT 32        /* feature width F (the only one supported) */
#define UNIGS_ANCHOR_HIDDEN 32      /* hidden width H of every MLP */
#define UNIGS_ANCHOR_MAX_OFFSETS 16 /* M: Gaussians per anchor, 1..16 */

/* One two-layer MLP, device, row-major float32: w1 [H][F], b1 [H],
 * w2 [out][H], b2 [out]. */
typedef struct {
    const float* w1;
    const float* b1;
    const float* w2;
    const float* b2;
} unigs_mlp;

/* The anchor set (device, float32): pos [3][n], scale [3][n] (> 0),
 * offsets [n][M][3], feat [n][F], sem [n][n_sem] (NULL when n_sem = 0),
 * kfac [n]; the five MLPs with out = n_sem, 1, M, 3M and 7M. */
typedef struct {
    int64_t n;
    int32_t n_offsets;  /* M */
    int32_t feat_dim;   /* must be UNIGS_ANCHOR_FEAT */
    int32_t hidden;     /* must be UNIGS_ANCHOR_HIDDEN */
    int32_t n_sem;      /* 0..UNIGS_MAX_SEM */
    const float* pos;
    const float* scale;
    const float* offsets;
    const float* feat;
    const float* sem;
    const float* kfac;
    unigs_mlp mlp_sem, mlp_k, mlp_opacity, mlp_color, mlp_cov;
} unigs_anchors;

/* Decoded Gaussians (device, caller-allocated, N = n M): mean [3][N],
 * quat [4][N], scale [3][N], opacity [N], kfac [N] float32; sh [N][1][3] and
 * sem [N][n_sem] float32 (feat_dtype 0) or bfloat16 (1, rounded to nearest
 * even).  Hand them to the rasterizer as a unigs_gaussians with n = N,
 * sh_degree 0, the same n_sem and feat_dtype. */
typedef struct {
    float* mean;
    float* quat;
    float* scale;
    float* opacity;
    float* kfac;
    void* sh;
    void* sem;
    int32_t feat_dtype;
    int32_t reserved;
} unigs_anchor_gaussians;

/* Forward: every anchor's M Gaussians (one thread per anchor, the MLP
 * weights in shared memory).  Returns UNIGS_ERR_INVALID_ARG for a NULL
 * pointer, n < 0, n_offsets outside 1..UNIGS_ANCHOR_MAX_OFFSETS, feat_dim or
 * hidden other than the supported widths, n_sem outside 0..UNIGS_MAX_SEM, or
 * feat_dtype other than 0 / 1. */
unigs_status unigs_anchor_decode(const unigs_anchors* a, const unigs_anchor_gaussians* out,
                                 unigs_stream stream);

/* Gradients of the anchor set, laid out like it (device, float32). */
typedef struct {
    float* w1;
    float* b1;
    float* w2;
    float* b2;
} unigs_mlp_grads;

typedef struct {
    float* pos;
    float* scale;
    float* offsets;
    float* feat;
    float* sem;
    float* kfac;
    unigs_mlp_grads mlp_sem, mlp_k, mlp_opacity, mlp_color, mlp_cov;
    int32_t accumulate; /* 0 overwrites, 1 adds to the existing contents */
    int32_t reserved;
} unigs_anchor_grads;

/* Backward of unigs_anchor_decode: from the decoded Gaussians' parameter
 * gradients (the unigs_param_grads of unigs_render_bwd; sh [N][1][3]),
 * dL/d(every anchor array and MLP parameter).  The per-anchor gradients are
 * written by one thread each; the MLP parameter gradients are summed over
 * blocks of 128 anchors in shared memory and added with one float32 atomic
 * per parameter and block (with accumulate = 0 they are cleared first).
 * NULL upstream arrays mean zero.  Same argument checks as the forward. */
unigs_status unigs_anchor_decode_bwd(const unigs_anchors* a, const unigs_param_grads* g,
                                     const unigs_anchor_grads* out, unigs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* UNIGS_ANCHORS_H */
