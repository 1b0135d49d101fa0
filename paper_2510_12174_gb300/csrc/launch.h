// Host-side launchers of the libunigs kernels (internal).
#pragma once

#include "unigs_internal.cuh"
#include "unigs_train.h"

namespace unigs {

// Each launcher returns the number of kernel launches it enqueued.
int launch_preprocess(const unigs_plan& p, const unigs_gaussians& g, const CamTable& tab,
                      void* ws, cudaStream_t st);
int launch_bin_sort(const unigs_plan& p, void* ws, cudaStream_t st);
int launch_render_fwd(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                      const unigs_outputs& out, cudaStream_t st);
// Tensor-core logit blend variant of the forward (bfloat16 logits, 9..64).
bool fwd_tc_eligible(const unigs_plan& p, const unigs_gaussians& g);
// Backward composite on the tensor cores: bfloat16 logits (9..64 channels),
// no UNIGS_FLAG_SIMT_LOGITS, launch shape default or batch 16 x 2 CTAs/SM.
bool bwd_tc_selected(const unigs_plan& p);
int launch_render_bwd_tc(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                         const unigs_outputs& fwd, const unigs_grad_outputs& go,
                         const unigs_param_grads& grads, double* grec, cudaStream_t st);
// Whether a float32 copy of bfloat16 logit rows is made per step: only the
// FP32-pipe composites read it.
bool sem32_needed(const unigs_plan& p);
int launch_render_fwd_tc(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                         const unigs_outputs& out, cudaStream_t st);
int launch_depth_normal_fwd(const unigs_plan& p, const CamTable& tab, const float* depth,
                            float* normal_d, cudaStream_t st);
int launch_depth_normal_bwd(const unigs_plan& p, const CamTable& tab, const float* depth,
                            const float* g_normal_d, const float* g_depth_in,
                            float* g_depth_out, cudaStream_t st);
int launch_render_bwd(const unigs_plan& p, const unigs_gaussians& g, void* ws,
                      const unigs_outputs& fwd, const unigs_grad_outputs& go,
                      const unigs_param_grads& grads, cudaStream_t st);

// One stable LSD radix pass over the n = hdr->n_instances pairs (n read on
// the device; 0 when hdr->status reports a capacity overflow) on the digit
// (key >> shift) & dmask (dmask 255 for a whole byte, 2^b - 1 to sort by b < 8
// bits): per-block digit histograms, their exclusive scan, stable scatter.  nb
// blocks of SORT_ITEMS pairs; hist holds 256 * nb counters, scan_tmp the scan
// partials.
int radix_pass(const unsigned long long* kin, const uint32_t* vin, unsigned long long* kout,
               uint32_t* vout, uint32_t* hist, uint32_t* scan_tmp, const WsHeader* hdr,
               int shift, uint32_t dmask, int nb, cudaStream_t st);

// Exclusive scan of n uint32 (three launches); partial holds
// ceil(n / SCAN_ITEMS) counters; *total (optional, device) gets the sum.
int scan_u32(const uint32_t* in, int64_t n, uint32_t* partial, uint32_t* out, uint32_t* total,
             cudaStream_t st);

// Training step (losses, Adam, pruning).
int launch_loss(const unigs_plan& p, const unigs_outputs& out, const float* normal_d,
                const unigs_targets& tgt, const unigs_loss_lambda& lam, void* ws, float* record,
                const unigs_loss_grads& g, cudaStream_t st);
int launch_adam(const unigs_adam_group* groups, int n_groups, const unigs_adam_hparams& hp,
                int32_t* step, cudaStream_t st);
int launch_param_copies(const unigs_adam_group* groups, int n_groups, cudaStream_t st);
size_t prune_ws_bytes(int64_t n);
int launch_prune_mark(const float* k, int64_t n, float T_k, void* ws, cudaStream_t st);
uint32_t* prune_count_ptr(void* ws, int64_t n);
int launch_prune_compact(const unigs_prune_array* arrays, int n_arrays, int64_t n, int64_t n_keep,
                         const void* ws, cudaStream_t st);

// Number of SMs of the current device (queried once per device).
int sm_count();

// Raises the dynamic shared-memory limit of kernel `func` to `bytes` on the
// current device, once per (kernel, device); thread-safe.  Returns the CUDA
// error of the attribute call (cudaSuccess when it was already set).
cudaError_t ensure_smem_limit(const void* func, int bytes);

// Index of the buffer (0/1) that holds the sorted keys/values after the sort.
inline int sorted_buffer(const unigs_plan& p) { return p.sort_passes & 1; }

}  // namespace unigs
