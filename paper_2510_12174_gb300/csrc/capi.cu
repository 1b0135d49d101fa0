// C ABI of libunigs: plan, workspace layout, argument checks, entry points.
#include <string.h>

#include <map>
#include <atomic>
#include <mutex>
#include <set>
#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"

using namespace unigs;

namespace unigs {
int sm_count() {
    // per device; concurrent first calls store the same value
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int c = cached[dev].load(std::memory_order_relaxed);
    if (!c) {
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
            c = 152;
        cached[dev].store(c, std::memory_order_relaxed);
    }
    return c;
}

cudaError_t ensure_smem_limit(const void* func, int bytes) {
    static std::mutex mu;
    // (kernel, device) -> the largest limit set so far (kernels whose
    // shared memory depends on runtime sizes raise it when they need more)
    static std::map<std::pair<const void*, int>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(func, dev);
    const auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}
}  // namespace unigs

namespace {

// One NVTX range per entry point (host side: it brackets the launches the call
// enqueues, so a profiler timeline shows the stages by name).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool build_cam_table(const unigs_plan* p, const unigs_camera* cams, CamTable* tab) {
    memset(tab, 0, sizeof(*tab));
    for (int k = 0; k < p->n_cams; ++k) {
        const unigs_camera& c = cams[k];
        DevCam& d = tab->cam[k];
        d.width = c.width;
        d.height = c.height;
        const int tw = p->cfg.tile_w, th = p->cfg.tile_h;
        d.tiles_x = (c.width + tw - 1) / tw;
        d.tiles_y = (c.height + th - 1) / th;
        d.tile_w = tw;
        d.tile_h = th;
        d.tile_off = p->tile_offset[k];
        d.pix_off = p->pixel_offset[k];
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        memcpy(d.R_wc, c.R_wc, sizeof(d.R_wc));
        memcpy(d.t_wc, c.t_wc, sizeof(d.t_wc));
        memcpy(d.R_cw, c.R_cw, sizeof(d.R_cw));
        memcpy(d.C, c.C, sizeof(d.C));
        d.z_near = c.z_near;
        if ((int64_t)d.tiles_x * d.tiles_y != p->tile_offset[k + 1] - p->tile_offset[k])
            return false;  // cameras differ from the plan
        if ((int64_t)c.width * c.height != p->pixel_offset[k + 1] - p->pixel_offset[k])
            return false;
    }
    return true;
}

unigs_status cuda_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? UNIGS_OK : UNIGS_ERR_CUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

bool check_gauss(const unigs_plan* p, const unigs_gaussians* g) {
    if (!g || g->n != p->n || g->sh_degree != p->sh_degree || g->n_sem != p->n_sem ||
        g->feat_dtype != p->feat_dtype)
        return false;
    if (p->n == 0) return true;
    if (!g->mean || !g->quat || !g->scale || !g->opacity || !g->kfac || !g->sh) return false;
    if (p->n_sem > 0 && !g->sem) return false;
    return aligned16(g->mean) && aligned16(g->quat) && aligned16(g->scale) &&
           aligned16(g->opacity) && aligned16(g->kfac) && aligned16(g->sh) &&
           (p->n_sem == 0 || aligned16(g->sem));
}

}  // namespace

extern "C" {

void unigs_config_default(unigs_config* cfg) {
    if (!cfg) return;
    cfg->alpha_min = 1.f / 255.f;
    cfg->alpha_max = 0.99f;
    cfg->T_min = 1e-4f;
    cfg->lowpass = 0.3f;
    cfg->step1 = 1;
    cfg->step2 = 2;
    cfg->lambda = 0.5f;
    cfg->flags = 0;
    cfg->batch = 0;
    cfg->ctas_per_sm = 0;
    cfg->batch_fwd = 0;
    cfg->ctas_per_sm_fwd = 0;
    cfg->tile_w = 0;
    cfg->tile_h = 0;
}

unigs_status unigs_plan_init(unigs_plan* plan, const unigs_gaussians* g, const unigs_camera* cams,
                             int32_t n_cams, const unigs_config* cfg, int64_t instance_capacity) {
    if (!plan || !g || !cams) return UNIGS_ERR_INVALID_ARG;
    if (g->n < 0 || g->n > 0x7fffffffLL) return UNIGS_ERR_INVALID_ARG;
    if (n_cams < 1 || n_cams > UNIGS_MAX_CAMS) return UNIGS_ERR_INVALID_ARG;
    if (g->sh_degree < 0 || g->sh_degree > 3) return UNIGS_ERR_INVALID_ARG;
    if (g->n_sem < 0 || g->n_sem > UNIGS_MAX_SEM) return UNIGS_ERR_INVALID_ARG;
    if (g->feat_dtype != 0 && g->feat_dtype != 1) return UNIGS_ERR_INVALID_ARG;
    if (instance_capacity < 0 || instance_capacity > 0x7fffffffLL) return UNIGS_ERR_INVALID_ARG;
    memset(plan, 0, sizeof(*plan));
    if (cfg)
        plan->cfg = *cfg;
    else
        unigs_config_default(&plan->cfg);
    if (plan->cfg.step1 < 1 || plan->cfg.step1 > 4 || plan->cfg.step2 < 1 || plan->cfg.step2 > 4)
        return UNIGS_ERR_INVALID_ARG;
    // the backward restores T by dividing by 1 - alpha, alpha <= alpha_max
    // (comparisons written so that NaN fails them)
    if (!(plan->cfg.alpha_min >= 0.f && plan->cfg.alpha_min <= plan->cfg.alpha_max &&
          plan->cfg.alpha_max < 1.f) ||
        !(plan->cfg.T_min >= 0.f && plan->cfg.T_min < 1.f) ||
        !(plan->cfg.lowpass >= 0.f && plan->cfg.lowpass < 1e30f))
        return UNIGS_ERR_INVALID_ARG;
    if (plan->cfg.flags &
        ~(UNIGS_FLAG_CENTER_DEPTH | UNIGS_FLAG_SIMT_LOGITS | UNIGS_FLAG_CHECK_FINITE))
        return UNIGS_ERR_INVALID_ARG;
    if (plan->cfg.batch != 0 && plan->cfg.batch != 8 && plan->cfg.batch != 16 &&
        plan->cfg.batch != 32 && plan->cfg.batch != 64)
        return UNIGS_ERR_INVALID_ARG;
    if (plan->cfg.ctas_per_sm < 0 || plan->cfg.ctas_per_sm > 8) return UNIGS_ERR_INVALID_ARG;
    if (plan->cfg.batch_fwd != 0 && plan->cfg.batch_fwd != 16 && plan->cfg.batch_fwd != 32 &&
        plan->cfg.batch_fwd != 64)
        return UNIGS_ERR_INVALID_ARG;
    if (plan->cfg.ctas_per_sm_fwd < 0 || plan->cfg.ctas_per_sm_fwd > 8)
        return UNIGS_ERR_INVALID_ARG;
    if (plan->cfg.tile_w == 0 && plan->cfg.tile_h == 0) plan->cfg.tile_w = plan->cfg.tile_h = TILE;
    {
        // 256 pixels per tile (one per composite thread), rows of whole 8x4
        // warp blocks
        const int tw = plan->cfg.tile_w, th = plan->cfg.tile_h;
        if (!((tw == 16 && th == 16) || (tw == 8 && th == 32) || (tw == 32 && th == 8) ||
              (tw == 64 && th == 4)))
            return UNIGS_ERR_INVALID_ARG;
    }
    plan->n = g->n;
    plan->n_cams = n_cams;
    plan->n_sem = g->n_sem;
    plan->sh_degree = g->sh_degree;
    plan->feat_dtype = g->feat_dtype;
    int64_t tiles = 0, pixels = 0;
    for (int k = 0; k < n_cams; ++k) {
        const unigs_camera& c = cams[k];
        if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384)
            return UNIGS_ERR_INVALID_ARG;
        if (!(c.fx > 0.f) || !(c.fy > 0.f)) return UNIGS_ERR_INVALID_ARG;
        plan->tile_offset[k] = (int32_t)tiles;
        plan->pixel_offset[k] = pixels;
        tiles += (int64_t)((c.width + plan->cfg.tile_w - 1) / plan->cfg.tile_w) *
                 ((c.height + plan->cfg.tile_h - 1) / plan->cfg.tile_h);
        pixels += (int64_t)c.width * c.height;
    }
    if (tiles > 0x7fffffffLL) return UNIGS_ERR_INVALID_ARG;
    plan->tile_offset[n_cams] = (int32_t)tiles;
    plan->pixel_offset[n_cams] = pixels;
    plan->n_tiles = tiles;
    plan->n_pixels = pixels;
    const int64_t total = g->n * (int64_t)n_cams;
    // a (camera, Gaussian) pair index is 32 bits wide in the device lists (the
    // per-pair workspace, over 500 bytes a pair, bounds it far lower anyway)
    if (total >= ((int64_t)1 << 32)) return UNIGS_ERR_INVALID_ARG;
    int64_t cap = instance_capacity ? instance_capacity : 4 * total;
    if (cap > 0x7fffffffLL) cap = 0x7fffffffLL;
    plan->capacity = cap;
    int tile_bits = 0;
    while (((int64_t)1 << tile_bits) < tiles) ++tile_bits;
    plan->sort_passes = (32 + tile_bits + 7) / 8;

    const int64_t nb_sort = (cap + SORT_ITEMS - 1) / SORT_ITEMS;
    const int64_t nb_scan_t = (total + SCAN_ITEMS - 1) / SCAN_ITEMS;
    const int64_t nb_scan_h = (256 * nb_sort + SCAN_ITEMS - 1) / SCAN_ITEMS;
    size_t sizes[OFF_END];
    sizes[OFF_HDR] = sizeof(WsHeader);
    sizes[OFF_CAM] = sizeof(CamTable);
    sizes[OFF_REC] = sizeof(float) * REC_FLOATS * (size_t)total;
    sizes[OFF_RECT] = sizeof(uint2) * (size_t)total;
    sizes[OFF_TOUCH] = sizeof(uint32_t) * (size_t)total;
    sizes[OFF_OFFS] = sizeof(uint32_t) * (size_t)total;
    sizes[OFF_ZBITS] = sizeof(uint32_t) * (size_t)total;
    sizes[OFF_SCAN] = sizeof(uint32_t) * (size_t)(nb_scan_t > nb_scan_h ? nb_scan_t : nb_scan_h) + 64;
    sizes[OFF_KEYS0] = sizeof(unsigned long long) * (size_t)cap;
    sizes[OFF_KEYS1] = sizeof(unsigned long long) * (size_t)cap;
    sizes[OFF_VALS0] = sizeof(uint32_t) * (size_t)cap;
    sizes[OFF_VALS1] = sizeof(uint32_t) * (size_t)cap;
    sizes[OFF_HIST] = sizeof(uint32_t) * 256 * (size_t)nb_sort;
    sizes[OFF_RANGES] = sizeof(uint2) * (size_t)tiles;
    sizes[OFF_GREC] = sizeof(double) * GREC_FLOATS * (size_t)total;
    sizes[OFF_CULL] = sizeof(float) * CULL_FLOATS * (size_t)total;
    // float32 copy of bfloat16 semantic rows, refreshed by every preprocess
    // when an FP32-pipe composite will read it
    sizes[OFF_SEM32] = sem32_needed(*plan) ? sizeof(float) * (size_t)g->n * g->n_sem : 0;
    sizes[OFF_ORDER] = sizeof(uint32_t) * (size_t)tiles;
    sizes[OFF_LOSS] = sizeof(float) * 8 * (size_t)LOSS_MAX_BLOCKS;
    // per (camera, Gaussian): the short-axis row of the projected scaled axes
    // E^T J R_wc R S, from the preprocess's double-float chain (float4)
    sizes[OFF_VP] = sizeof(float) * 4 * (size_t)total;
    size_t off = 0;
    for (int r = 0; r < OFF_END; ++r) {
        plan->off[r] = off;
        off = align_up(off + sizes[r], 256);
    }
    plan->ws_bytes = off;
    return UNIGS_OK;
}

size_t unigs_workspace_bytes(const unigs_plan* plan) { return plan ? plan->ws_bytes : 0; }

unigs_status unigs_preprocess(const unigs_plan* plan, const unigs_gaussians* g,
                              const unigs_camera* cams, void* ws, unigs_stream stream) {
    NvtxRange nvtx_range("unigs_preprocess");
    if (!plan || !cams || !ws || !aligned16(ws) || !check_gauss(plan, g))
        return UNIGS_ERR_INVALID_ARG;
    static thread_local CamTable tab;
    if (!build_cam_table(plan, cams, &tab)) return UNIGS_ERR_INVALID_ARG;
    launch_preprocess(*plan, *g, tab, ws, (cudaStream_t)stream);
    return cuda_status();
}

unigs_status unigs_bin_sort(const unigs_plan* plan, void* ws, int64_t* n_instances_out,
                            unigs_stream stream) {
    NvtxRange nvtx_range("unigs_bin_sort");
    if (!plan || !ws || !aligned16(ws)) return UNIGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    launch_bin_sort(*plan, ws, st);
    unigs_status s = cuda_status();
    if (s != UNIGS_OK || !n_instances_out) return s;
    WsHeader h;
    if (cudaMemcpyAsync(&h, ws_ptr<WsHeader>(ws, *plan, OFF_HDR), 32, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return UNIGS_ERR_CUDA;
    *n_instances_out = (int64_t)h.need;
    if (h.status == UNIGS_ERR_CAPACITY) return UNIGS_ERR_CAPACITY;
    return (unigs_status)h.status;
}

unigs_status unigs_render_fwd(const unigs_plan* plan, const unigs_gaussians* g, void* ws,
                              const unigs_outputs* out, unigs_stream stream) {
    NvtxRange nvtx_range("unigs_render_fwd");
    if (!plan || !ws || !out || !check_gauss(plan, g)) return UNIGS_ERR_INVALID_ARG;
    if (!out->rgb || !out->depth || !out->normal_g || !out->kmap || !out->T_final ||
        !out->n_contrib || (plan->n_sem > 0 && !out->logits))
        return UNIGS_ERR_INVALID_ARG;
    launch_render_fwd(*plan, *g, ws, *out, (cudaStream_t)stream);
    return cuda_status();
}

unigs_status unigs_depth_normal_fwd(const unigs_plan* plan, const unigs_camera* cams,
                                    const float* depth, float* normal_d, unigs_stream stream) {
    NvtxRange nvtx_range("unigs_depth_normal_fwd");
    if (!plan || !cams || !depth || !normal_d) return UNIGS_ERR_INVALID_ARG;
    static thread_local CamTable tab;
    if (!build_cam_table(plan, cams, &tab)) return UNIGS_ERR_INVALID_ARG;
    launch_depth_normal_fwd(*plan, tab, depth, normal_d, (cudaStream_t)stream);
    return cuda_status();
}

unigs_status unigs_depth_normal_bwd(const unigs_plan* plan, const unigs_camera* cams,
                                    const float* depth, const float* g_normal_d,
                                    const float* g_depth_in, float* g_depth_out,
                                    unigs_stream stream) {
    NvtxRange nvtx_range("unigs_depth_normal_bwd");
    if (!plan || !cams || !depth || !g_normal_d || !g_depth_out) return UNIGS_ERR_INVALID_ARG;
    static thread_local CamTable tab;
    if (!build_cam_table(plan, cams, &tab)) return UNIGS_ERR_INVALID_ARG;
    launch_depth_normal_bwd(*plan, tab, depth, g_normal_d, g_depth_in, g_depth_out,
                            (cudaStream_t)stream);
    return cuda_status();
}

unigs_status unigs_render_bwd(const unigs_plan* plan, const unigs_gaussians* g,
                              const unigs_camera* cams, void* ws, const unigs_outputs* fwd,
                              const unigs_grad_outputs* grad_out, unigs_param_grads* grads,
                              unigs_stream stream) {
    NvtxRange nvtx_range("unigs_render_bwd");
    (void)cams;
    if (!plan || !ws || !fwd || !grad_out || !grads || !check_gauss(plan, g))
        return UNIGS_ERR_INVALID_ARG;
    if (!fwd->T_final || !fwd->n_contrib) return UNIGS_ERR_INVALID_ARG;
    if (plan->n_sem > 0 && !grads->sem) return UNIGS_ERR_INVALID_ARG;
    launch_render_bwd(*plan, *g, ws, *fwd, *grad_out, *grads, (cudaStream_t)stream);
    return cuda_status();
}

unigs_status unigs_status_poll(const unigs_plan* plan, const void* ws, int64_t* detail,
                               unigs_stream stream) {
    if (!plan || !ws) return UNIGS_ERR_INVALID_ARG;
    WsHeader h;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, ws_ptr<WsHeader>(const_cast<void*>(ws), *plan, OFF_HDR), 64,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return UNIGS_ERR_CUDA;
    if (detail)
        *detail = h.status == UNIGS_ERR_NONFINITE ? (int64_t)h.nonfinite : (int64_t)h.need;
    return (unigs_status)h.status;
}

unigs_status unigs_stats_poll(const unigs_plan* plan, const void* ws, int64_t* pairs_evaluated,
                              int64_t* pairs_blended, unigs_stream stream) {
    if (!plan || !ws) return UNIGS_ERR_INVALID_ARG;
    WsHeader h;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, ws_ptr<WsHeader>(const_cast<void*>(ws), *plan, OFF_HDR), 64,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return UNIGS_ERR_CUDA;
    if (pairs_evaluated) *pairs_evaluated = (int64_t)h.n_eval;
    if (pairs_blended) *pairs_blended = (int64_t)h.n_blend;
    return UNIGS_OK;
}

int32_t unigs_launches_per_step(const unigs_plan* plan) {
    if (!plan) return 0;
    const int per_pass = 1 + 3 + 1;
    const int bin = 3 + 1 + per_pass * plan->sort_passes + 1 + 1 /*tile order*/;
    int conv = 0;
    if (sem32_needed(*plan)) {
        const int64_t cnt = plan->n * (int64_t)plan->n_sem;
        conv = (cnt / 2 > 0 ? 1 : 0) + (int)(cnt & 1);
    }
    const int check = (plan->cfg.flags & UNIGS_FLAG_CHECK_FINITE) && plan->n > 0 ? 1 : 0;
    return 3 /*preprocess: init, culling pass, splat pass*/ + check + conv + bin + 1 /*fwd*/ + 1 /*dn fwd*/ + 1 /*dn bwd*/ +
           3 /*bwd: record zeroing, composite, preprocess bwd*/;
}

int32_t unigs_plan_paths(const unigs_plan* plan) {
    if (!plan) return 0;
    int32_t bits = 0;
    if (plan->n_sem >= 9 && plan->n_sem <= UNIGS_MAX_SEM &&
        !(plan->cfg.flags & UNIGS_FLAG_SIMT_LOGITS))
        bits |= UNIGS_PATH_FWD_TC;
    if (bwd_tc_selected(*plan)) bits |= UNIGS_PATH_BWD_TC;
    if (sem32_needed(*plan)) bits |= UNIGS_PATH_SEM32;
    return bits;
}

// ------------------------------------------------------------ training step
void unigs_loss_lambda_default(unigs_loss_lambda* lam) {
    if (!lam) return;
    lam->l1 = 1.f;
    lam->normal = lam->depth = lam->seg = lam->K = 0.1f;
}

unigs_status unigs_loss(const unigs_plan* plan, const unigs_outputs* out, const float* normal_d,
                        const unigs_targets* tgt, const unigs_loss_lambda* lambda, void* ws,
                        float* record, const unigs_loss_grads* grads, unigs_stream stream) {
    NvtxRange nvtx_range("unigs_loss");
    if (!plan || !out || !tgt || !lambda || !ws || !record || !grads) return UNIGS_ERR_INVALID_ARG;
    if ((tgt->rgb && !out->rgb) || (tgt->depth && !out->depth) || (tgt->normal && !normal_d) ||
        (tgt->label && (!out->logits || plan->n_sem == 0)))
        return UNIGS_ERR_INVALID_ARG;
    launch_loss(*plan, *out, normal_d, *tgt, *lambda, ws, record, *grads, (cudaStream_t)stream);
    return cuda_status();
}

unigs_status unigs_adam_step(const unigs_adam_group* groups, int32_t n_groups,
                             const unigs_adam_hparams* hp, int32_t* step, unigs_stream stream) {
    NvtxRange nvtx_range("unigs_adam_step");
    if (!hp || !step || n_groups < 0 || n_groups > UNIGS_ADAM_MAX_GROUPS ||
        (n_groups > 0 && !groups))
        return UNIGS_ERR_INVALID_ARG;
    for (int i = 0; i < n_groups; ++i) {
        const unigs_adam_group& G = groups[i];
        if (G.count < 0 || G.activation < UNIGS_ACT_NONE || G.activation > UNIGS_ACT_SIGMOID)
            return UNIGS_ERR_INVALID_ARG;
        if (G.count > 0 && (!G.param || !G.grad || !G.m || !G.v)) return UNIGS_ERR_INVALID_ARG;
        if (G.act_out == G.param && G.activation != UNIGS_ACT_NONE) return UNIGS_ERR_INVALID_ARG;
    }
    launch_adam(groups, n_groups, *hp, step, (cudaStream_t)stream);
    return cuda_status();
}

unigs_status unigs_param_copies(const unigs_adam_group* groups, int32_t n_groups,
                                unigs_stream stream) {
    NvtxRange nvtx_range("unigs_param_copies");
    if (n_groups < 0 || n_groups > UNIGS_ADAM_MAX_GROUPS || (n_groups > 0 && !groups))
        return UNIGS_ERR_INVALID_ARG;
    for (int i = 0; i < n_groups; ++i) {
        const unigs_adam_group& G = groups[i];
        if (G.count < 0 || G.activation < UNIGS_ACT_NONE || G.activation > UNIGS_ACT_SIGMOID)
            return UNIGS_ERR_INVALID_ARG;
        if (G.count > 0 && !G.param) return UNIGS_ERR_INVALID_ARG;
        if (G.act_out == G.param && G.activation != UNIGS_ACT_NONE) return UNIGS_ERR_INVALID_ARG;
    }
    launch_param_copies(groups, n_groups, (cudaStream_t)stream);
    return cuda_status();
}

size_t unigs_prune_workspace_bytes(int64_t n) { return n < 0 ? 0 : prune_ws_bytes(n); }

unigs_status unigs_prune_mark(const float* k, int64_t n, float T_k, void* prune_ws,
                              int64_t* n_keep, unigs_stream stream) {
    NvtxRange nvtx_range("unigs_prune_mark");
    if (n < 0 || n > 0xffffffffLL || (n > 0 && !k) || !prune_ws || !aligned16(prune_ws) || !n_keep)
        return UNIGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    launch_prune_mark(k, n, T_k, prune_ws, st);
    unigs_status s = cuda_status();
    if (s != UNIGS_OK) return s;
    uint32_t cnt = 0;
    if (cudaMemcpyAsync(&cnt, prune_count_ptr(prune_ws, n), sizeof(cnt), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return UNIGS_ERR_CUDA;
    *n_keep = (int64_t)cnt;
    return UNIGS_OK;
}

unigs_status unigs_prune_compact(const unigs_prune_array* arrays, int32_t n_arrays, int64_t n,
                                 int64_t n_keep, const void* prune_ws, unigs_stream stream) {
    NvtxRange nvtx_range("unigs_prune_compact");
    if (n < 0 || n_keep < 0 || n_keep > n || n_arrays < 0 || (n_arrays > 0 && !arrays) ||
        !prune_ws)
        return UNIGS_ERR_INVALID_ARG;
    for (int a = 0; a < n_arrays; ++a) {
        const unigs_prune_array& A = arrays[a];
        if (A.planes < 1 || A.row < 1 || (A.elem_bytes != 4 && A.elem_bytes != 2) ||
            (A.fill && A.elem_bytes != 4) || (!A.fill && n > 0 && !A.src) ||
            (n_keep > 0 && !A.dst) || (A.src && A.src == A.dst))
            return UNIGS_ERR_INVALID_ARG;
    }
    launch_prune_compact(arrays, n_arrays, n, n_keep, prune_ws, (cudaStream_t)stream);
    return cuda_status();
}

const char* unigs_status_string(unigs_status s) {
    switch (s) {
        case UNIGS_OK: return "ok";
        case UNIGS_ERR_INVALID_ARG: return "invalid argument";
        case UNIGS_ERR_CAPACITY: return "instance capacity exceeded";
        case UNIGS_ERR_CUDA: return "CUDA error";
        case UNIGS_ERR_NONFINITE: return "non-finite value";
        case UNIGS_ERR_TIMEOUT: return "bounded device wait timed out";
    }
    return "unknown status";
}

}  // extern "C"
