/*
 * unigs_train.h - C ABI of the training step around the rasterizer (sm_103a).
 *
 * The combined objective of Sec. 3.4 ("Loss Function") without its SSIM term,
 * the Adam update of the Gaussian parameters with float32 master values and
 * bfloat16 feature copies, and the k-pruning rule of Sec. 3.3 ("Pruning").
 * Conventions (device/host pointers, streams, the concatenated multi-camera
 * image layout, status codes) are those of unigs.h.
 */
#ifndef UNIGS_TRAIN_H
#define UNIGS_TRAIN_H

#include "unigs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ losses */

/* Targets of the objective (device, the concatenated layout of the outputs):
 * rgb 3 channels; depth 1 channel, values <= 0 mark pixels without a
 * measurement (left out of L_depth); normal 3 channels, the target of the
 * normal-from-depth map; label 1 channel of int32 class ids, values outside
 * [0, n_sem) mark unlabelled pixels (left out of L_seg).  A NULL pointer
 * drops its term (weight 0). */
typedef struct {
    const float* rgb;
    const float* depth;
    const float* normal;
    const int32_t* label;
} unigs_targets;

/* lambda of Sec. 3.4: l1 weighs L_l1 directly, the others scale the
 * magnitude-normalised terms lambda_i * |L_l1| * L_i / |L_i|.  The paper sets
 * lambda_1 = 1 and every other lambda 0.1 (unigs_loss_lambda_default). */
typedef struct {
    float l1, normal, depth, seg, K;
} unigs_loss_lambda;

void unigs_loss_lambda_default(unigs_loss_lambda* lam);

/* Loss record, device float[UNIGS_LOSS_RECORD_FLOATS], written by
 * unigs_loss: the total, the five term values, their weights
 * (w_l1 = lambda_1; w_i = lambda_i |L_l1| / |L_i|, 0 when L_i = 0) and the
 * pixel counts of the depth and segmentation terms. */
enum {
    UNIGS_LOSS_TOTAL = 0,
    UNIGS_LOSS_L1 = 1, UNIGS_LOSS_NORMAL, UNIGS_LOSS_DEPTH, UNIGS_LOSS_SEG, UNIGS_LOSS_K,
    UNIGS_LOSS_W_L1 = 6, UNIGS_LOSS_W_NORMAL, UNIGS_LOSS_W_DEPTH, UNIGS_LOSS_W_SEG, UNIGS_LOSS_W_K,
    UNIGS_LOSS_N_DEPTH = 11, UNIGS_LOSS_N_LABEL = 12,
    UNIGS_LOSS_RECORD_FLOATS = 16
};

/* dL_all/d(rendered map), device, the layouts of the outputs.  NULL entries
 * are not written. */
typedef struct {
    float* rgb;
    float* depth;    /* the L_depth part only: pass it as g_depth_in of
                        unigs_depth_normal_bwd together with normal_d */
    float* normal_d;
    float* kmap;
    float* logits;
} unigs_loss_grads;

/* The five terms over the pixels of all cameras of the plan, with
 * P = plan->n_pixels:
 *   L_l1     = sum |rgb - rgb_t| / (3 P)
 *   L_normal = 1 - sum normal_d . normal_t / P        (Eq. csloss, the mean
 *              over Omega = every pixel; gradient -normal_t / P, Eq. gradientn)
 *   L_depth  = sum over measured pixels |depth - depth_t| / (their count)
 *   L_seg    = mean over labelled pixels of -log softmax(logits)[label]
 *   L_K      = sum |kmap - 1| / P                      (Sec. 3.3, L_K)
 * then L_all = w_l1 L_l1 + sum_i w_i L_i with the weights of the record
 * treated as constants of the step, and the gradients of L_all (the L1
 * subgradient is 0 at 0).  out supplies rgb, depth, kmap and logits;
 * normal_d is the map of unigs_depth_normal_fwd.  Uses the workspace's loss
 * region (plan from unigs_plan_init).  Three launches, no synchronisation
 * (graph-capturable).  UNIGS_ERR_INVALID_ARG for a NULL record or a target
 * without its output. */
unigs_status unigs_loss(const unigs_plan* plan, const unigs_outputs* out, const float* normal_d,
                        const unigs_targets* tgt, const unigs_loss_lambda* lambda, void* ws,
                        float* record, const unigs_loss_grads* grads, unigs_stream stream);

/* ------------------------------------------------------------------- Adam */

typedef enum {
    UNIGS_ACT_NONE = 0,   /* the renderer reads the raw value               */
    UNIGS_ACT_EXP = 1,    /* scales: the renderer reads exp(raw)            */
    UNIGS_ACT_SIGMOID = 2 /* opacity: the renderer reads 1 / (1 + exp(-raw)) */
} unigs_activation;

/* One parameter array.  param holds the raw float32 master values (updated
 * in place); grad is dL/d(activated value) as unigs_render_bwd writes it
 * (the update multiplies by the activation's derivative at the raw value);
 * m, v the Adam moments.  act_out (optional) receives the activated float32
 * value after the update, bf16_out (optional) its bfloat16 rounding (to
 * nearest even) - the copies the renderer reads. */
typedef struct {
    float* param;
    const float* grad;
    float* m;
    float* v;
    float* act_out;
    void* bf16_out;
    int64_t count;
    float lr;
    int32_t activation;
} unigs_adam_group;

typedef struct {
    float beta1, beta2, eps;
} unigs_adam_hparams;

#define UNIGS_ADAM_MAX_GROUPS 16

/* Adam (Kingma & Ba 2015, Algorithm 1; the paper trains with LibTorch without
 * naming its optimizer, and Adam is the one of the 3DGS pipeline it extends)
 * over up to UNIGS_ADAM_MAX_GROUPS arrays in one launch.  step is a
 * device int32 counter: the update uses t = *step + 1 for the bias
 * corrections and a second launch stores t (graph-capturable).  groups and
 * hp are host memory.  UNIGS_ERR_INVALID_ARG for NULL param/grad/m/v, a
 * negative count, an unknown activation, or act_out == param with an
 * activation. */
unigs_status unigs_adam_step(const unigs_adam_group* groups, int32_t n_groups,
                             const unigs_adam_hparams* hp, int32_t* step, unigs_stream stream);

/* The activated float32 and bfloat16 copies of each group's raw values, as
 * unigs_adam_step writes them after an update, without an update (grad, m,
 * v, lr ignored): after a prune or a checkpoint load.  Same argument checks
 * (grad, m, v may be NULL). */
unigs_status unigs_param_copies(const unigs_adam_group* groups, int32_t n_groups,
                                unigs_stream stream);

/* ---------------------------------------------------------------- pruning */

size_t unigs_prune_workspace_bytes(int64_t n);

/* Pruning rule of Sec. 3.3: Gaussian i survives when |k_i - 1| <= T_k
 * (float32 comparison).  Marks the survivors and scans their positions in
 * prune_ws (unigs_prune_workspace_bytes(n) bytes, device); *n_keep (host)
 * receives the survivor count, which synchronises the stream. */
unigs_status unigs_prune_mark(const float* k, int64_t n, float T_k, void* prune_ws,
                              int64_t* n_keep, unigs_stream stream);

/* One array to compact: planes x n rows of row elements of elem_bytes (4 or
 * 2) bytes, plane-major (SoA [planes][n][row]; planes = 1 for row-major
 * [n][row]).  dst holds planes x n_keep rows and must not overlap src.  With
 * fill != 0 every surviving element is set to fill_value instead of copied
 * (the reset of k to 0.9 after a prune, and of its Adam moments to 0; 4-byte
 * elements only). */
typedef struct {
    const void* src;
    void* dst;
    int32_t planes;
    int32_t row;
    int32_t elem_bytes;
    int32_t fill;
    float fill_value;
    int32_t reserved;
} unigs_prune_array;

/* Copies the survivors of the last unigs_prune_mark on prune_ws, in their
 * original order, from every src to its dst.  n and n_keep as in that call. */
unigs_status unigs_prune_compact(const unigs_prune_array* arrays, int32_t n_arrays, int64_t n,
                                 int64_t n_keep, const void* prune_ws, unigs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* UNIGS_TRAIN_H */
