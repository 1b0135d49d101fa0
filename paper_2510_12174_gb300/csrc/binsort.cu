// Binning: scan of tiles touched, key emission, stable LSD radix sort, ranges.
//
// The paper extends the tile pipeline of 3DGS (Sec. 3.4): each Gaussian is
// duplicated once per tile its 3-sigma rectangle overlaps, keyed by
// (global tile id << 32 | float32 bits of its camera-frame centre depth), and
// the keys are sorted so that every tile holds a front-to-back list.  Depths
// are > z_near > 0, so their bit patterns order like the values.  The sort is
// a stable LSD radix sort over the used key bits (8-bit digits), so ties in
// depth keep the emission order (Gaussian index): the order within a tile is
// (depth, index).
//
// Every kernel reads the instance count from the workspace header, so the
// whole sequence runs without a host round trip (CUDA-graph capture); grids
// are sized from the plan's capacity and surplus blocks exit at once.
#include "launch.h"

namespace unigs {

// ------------------------------------------------------------ block scan
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh_warp,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? sh_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh_warp[lane] = s;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const uint32_t warp_base = wid ? sh_warp[wid - 1] : 0;
    if (total) *total = sh_warp[(blockDim.x >> 5) - 1];
    const uint32_t r = warp_base + x - v;
    __syncthreads();
    return r;
}

// Phase 1: per-block sums of SCAN_ITEMS elements.
__global__ void __launch_bounds__(256)
    scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ partial) {
    __shared__ uint32_t sw[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
    for (int j = threadIdx.x; j < SCAN_ITEMS; j += blockDim.x) {
        const int64_t i = base + j;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_exclusive_scan(s, sw, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Phase 2: exclusive scan of the block sums by one block; writes the total.
__global__ void __launch_bounds__(1024)
    scan_partials_kernel(uint32_t* __restrict__ partial, int64_t nb, uint32_t* __restrict__ total_out) {
    __shared__ uint32_t sw[32];
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const uint32_t v = i < nb ? partial[i] : 0;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, sw, &tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

// Phase 3: scan within each block, offset by the scanned block sum.
__global__ void __launch_bounds__(256)
    scan_down_kernel(const uint32_t* __restrict__ in, int64_t n, const uint32_t* __restrict__ partial,
                     uint32_t* __restrict__ out) {
    __shared__ uint32_t sw[32];
    constexpr int PER = SCAN_ITEMS / 256;
    const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS + (int64_t)threadIdx.x * PER;
    uint32_t v[PER];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int64_t i = base + j;
        v[j] = i < n ? in[i] : 0;
        s += v[j];
    }
    uint32_t run = block_exclusive_scan(s, sw, nullptr) + partial[blockIdx.x];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int64_t i = base + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
}

int scan_u32(const uint32_t* in, int64_t n, uint32_t* partial, uint32_t* out, uint32_t* total,
             cudaStream_t st) {
    const int64_t nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
    if (nb == 0) return 0;
    scan_reduce_kernel<<<(unsigned)nb, 256, 0, st>>>(in, n, partial);
    scan_partials_kernel<<<1, 1024, 0, st>>>(partial, nb, total);
    scan_down_kernel<<<(unsigned)nb, 256, 0, st>>>(in, n, partial, out);
    return 3;
}

// ------------------------------------------------------------ emission
// Total = offsets[last] + touched[last]; checks the capacity and writes one
// (key, value) per overlapped tile in (camera, Gaussian, tile row-major)
// order.
__global__ void __launch_bounds__(256)
    emit_kernel(const CamTable* __restrict__ tab, int64_t n, int n_cams, int tw, int th,
                int64_t capacity,
                const uint2* __restrict__ rect, const uint32_t* __restrict__ touched,
                const uint32_t* __restrict__ offs, const uint32_t* __restrict__ zbits,
                const float* __restrict__ cull, WsHeader* __restrict__ hdr,
                unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t total = n * (int64_t)n_cams;
    const uint64_t need = (uint64_t)offs[total - 1] + touched[total - 1];
    if (need > (uint64_t)capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            hdr->need = need;
            hdr->n_instances = 0;
            set_status(hdr, UNIGS_ERR_CAPACITY);
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hdr->n_instances = (uint32_t)need;
        hdr->need = need;
    }
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    // uniform loop bound: whole warps iterate together, so rectangles larger
    // than 32 tiles are emitted cooperatively (ballot compaction keeps the
    // row-major order)
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const uint32_t cnt = t < total ? touched[t] : 0u;
        int x0 = 0, x1 = 0, y0 = 0, y1 = 0, k = 0;
        uint32_t g = 0, o = 0;
        unsigned long long zb = 0, toff = 0;
        int tiles_x = 0;
        float cr[CULL_FLOATS] = {};
        if (cnt) {
            k = (int)(t / n);
            g = (uint32_t)(t - (int64_t)k * n);
            const DevCam& cam = tab->cam[k];
            const uint2 r = rect[t];
            x0 = r.x & 0xffff; x1 = r.x >> 16; y0 = r.y & 0xffff; y1 = r.y >> 16;
            zb = zbits[t];
            toff = (unsigned long long)cam.tile_off;
            tiles_x = cam.tiles_x;
            o = offs[t];
            const float4* src = reinterpret_cast<const float4*>(cull + (size_t)t * CULL_FLOATS);
            const float4 c0 = src[0], c1 = src[1];
            cr[0] = c0.x; cr[1] = c0.y; cr[2] = c0.z; cr[3] = c0.w;
            cr[4] = c1.x; cr[5] = c1.y; cr[6] = c1.z; cr[7] = c1.w;
        }
        const int nt = (x1 - x0) * (y1 - y0);
        if (cnt && nt <= COOP_TILES) {
            const uint32_t o_end = o + cnt;
            for (int ty = y0; ty < y1; ++ty)
                for (int tx = x0; tx < x1; ++tx) {
                    if (!tile_keep(cr, tx, ty, tw, th) || o >= o_end) continue;
                    const unsigned long long tile = toff + (unsigned long long)(ty * tiles_x + tx);
                    keys[o] = (tile << 32) | zb;
                    vals[o] = g;
                    ++o;
                }
        }
        unsigned big = __ballot_sync(0xffffffffu, cnt && nt > COOP_TILES);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            float cb[CULL_FLOATS];
#pragma unroll
            for (int q = 0; q < CULL_FLOATS; ++q) cb[q] = __shfl_sync(0xffffffffu, cr[q], src);
            const int bx0 = __shfl_sync(0xffffffffu, x0, src);
            const int by0 = __shfl_sync(0xffffffffu, y0, src);
            const int bw = __shfl_sync(0xffffffffu, x1 - x0, src);
            const int bn = __shfl_sync(0xffffffffu, nt, src);
            const int btx = __shfl_sync(0xffffffffu, tiles_x, src);
            const unsigned long long btoff = __shfl_sync(0xffffffffu, toff, src);
            const unsigned long long bzb = __shfl_sync(0xffffffffu, zb, src);
            const uint32_t bg = __shfl_sync(0xffffffffu, g, src);
            uint32_t bo = __shfl_sync(0xffffffffu, o, src);
            const uint32_t bend = bo + __shfl_sync(0xffffffffu, cnt, src);
            for (int j0 = 0; j0 < bn; j0 += 32) {
                const int j = j0 + lane;
                const int tx = bx0 + j % bw, ty = by0 + j / bw;
                const bool keep = j < bn && tile_keep(cb, tx, ty, tw, th);
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                const uint32_t dst = bo + __popc(m & lt_mask);
                if (keep && dst < bend) {
                    const unsigned long long tile = btoff + (unsigned long long)(ty * btx + tx);
                    keys[dst] = (tile << 32) | bzb;
                    vals[dst] = bg;
                }
                bo += __popc(m);
            }
        }
    }
}

// ------------------------------------------------------------ radix sort
__device__ __forceinline__ uint32_t n_valid(const WsHeader* hdr) {
    return hdr->status == UNIGS_ERR_CAPACITY ? 0u : hdr->n_instances;
}

// Per-block digit counts, stored digit-major: hist[d * nb + b].  The digit of
// a key is (key >> shift) & dmask (dmask 255 for a whole byte; fewer bits on
// a last pass that must ignore the key bits above the sorted ones).
__global__ void __launch_bounds__(256)
    radix_hist_kernel(const unsigned long long* __restrict__ keys, const WsHeader* __restrict__ hdr,
                      int shift, uint32_t dmask, int nb, uint32_t* __restrict__ hist) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t n = n_valid(hdr);
    const int64_t base = (int64_t)blockIdx.x * SORT_ITEMS;
    for (int j = threadIdx.x; j < SORT_ITEMS; j += 256) {
        const int64_t i = base + j;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & dmask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter.  Warp w of the block owns keys [w*256, w*256+256) of the
// block's chunk and walks them 32 at a time in order; __match_any_sync ranks
// equal digits inside each step, a per-warp running count orders the steps,
// and a prefix over warps orders the warps.  The block's pairs are first
// placed in shared memory in (digit, input order) order, then written out by
// consecutive threads: the pairs of one digit land at consecutive addresses,
// so the stores coalesce.
__global__ void __launch_bounds__(256)
    radix_scatter_kernel(const unsigned long long* __restrict__ kin,
                         const uint32_t* __restrict__ vin, unsigned long long* __restrict__ kout,
                         uint32_t* __restrict__ vout, const uint32_t* __restrict__ scanned,
                         const WsHeader* __restrict__ hdr, int shift, uint32_t dmask, int nb) {
    __shared__ uint32_t whist[8][256];
    __shared__ uint32_t goff[256];
    __shared__ uint32_t loff[256];  // first block-local position of each digit
    __shared__ uint32_t wsum[8];
    __shared__ unsigned long long sk[SORT_ITEMS];
    __shared__ uint32_t sv[SORT_ITEMS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < 8 * 256; j += 256) (&whist[0][0])[j] = 0;
    goff[threadIdx.x] = scanned[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();
    const uint32_t n = n_valid(hdr);
    const int64_t block0 = (int64_t)blockIdx.x * SORT_ITEMS;
    const int64_t base = block0 + w * 256;
    const uint32_t lt_mask = (1u << lane) - 1u;
    unsigned long long k[8];
    uint32_t v[8], rank[8], dig[8];
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int64_t i = base + it * 32 + lane;
        const bool ok = i < n;
        k[it] = ok ? kin[i] : 0ull;
        v[it] = ok ? vin[i] : 0u;
        const uint32_t d = ok ? ((uint32_t)(k[it] >> shift) & dmask) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = (d < 256u) ? whist[w][d] : 0u;
        __syncwarp();
        if (d < 256u && lane == __ffs(peers) - 1) whist[w][d] = before + __popc(peers);
        __syncwarp();
        rank[it] = before + __popc(peers & lt_mask);
        dig[it] = d;
    }
    __syncthreads();
    {
        // per digit: the warps' exclusive offsets within the digit, then an
        // exclusive scan of the digit totals over the block
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w2 = 0; w2 < 8; ++w2) {
            const uint32_t c = whist[w2][d];
            whist[w2][d] = run;
            run += c;
        }
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t wp = 0;
        for (int w2 = 0; w2 < w; ++w2) wp += wsum[w2];
        loff[d] = wp + x - run;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const uint32_t d = dig[it];
        if (d < 256u) {
            const uint32_t lp = loff[d] + whist[w][d] + rank[it];
            sk[lp] = k[it];
            sv[lp] = v[it];
        }
    }
    __syncthreads();
    // the valid pairs are a prefix of the block's chunk
    const int64_t rem = (int64_t)n - block0;
    const int cnt = rem <= 0 ? 0 : (rem < SORT_ITEMS ? (int)rem : SORT_ITEMS);
    for (int j = threadIdx.x; j < cnt; j += 256) {
        const unsigned long long key = sk[j];
        const uint32_t d = (uint32_t)(key >> shift) & dmask;
        const uint32_t dst = goff[d] + ((uint32_t)j - loff[d]);
        kout[dst] = key;
        vout[dst] = sv[j];
    }
}

// Per-tile [start, end) by boundary detection on the sorted keys.
__global__ void __launch_bounds__(256)
    ranges_kernel(const unsigned long long* __restrict__ keys, const WsHeader* __restrict__ hdr,
                  uint2* __restrict__ ranges) {
    const uint32_t n = n_valid(hdr);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
        if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

// Tile schedule of the persistent composite kernels: global tile ids ordered
// by descending list length, bucketed by floor(log2(length)) (one block;
// the order inside a bucket is arbitrary and affects scheduling only).
__global__ void __launch_bounds__(1024)
    tile_order_kernel(const uint2* __restrict__ ranges, int64_t n_tiles, uint32_t* __restrict__ order) {
    __shared__ uint32_t cnt[33];
    __shared__ uint32_t base[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        atomicAdd(&cnt[__clz(r.y - r.x)], 1u);  // longer lists -> fewer leading zeros
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < 33; ++b) {
            base[b] = run;
            run += cnt[b];
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        order[atomicAdd(&base[__clz(r.y - r.x)], 1u)] = (uint32_t)t;
    }
}

int radix_pass(const unsigned long long* kin, const uint32_t* vin, unsigned long long* kout,
               uint32_t* vout, uint32_t* hist, uint32_t* scan_tmp, const WsHeader* hdr,
               int shift, uint32_t dmask, int nb, cudaStream_t st) {
    radix_hist_kernel<<<nb, 256, 0, st>>>(kin, hdr, shift, dmask, nb, hist);
    int launches = 1 + scan_u32(hist, (int64_t)nb * 256, scan_tmp, hist, nullptr, st);
    radix_scatter_kernel<<<nb, 256, 0, st>>>(kin, vin, kout, vout, hist, hdr, shift, dmask, nb);
    return launches + 1;
}

int launch_bin_sort(const unigs_plan& p, void* ws, cudaStream_t st) {
    const int64_t total = p.n * (int64_t)p.n_cams;
    WsHeader* hdr = ws_ptr<WsHeader>(ws, p, OFF_HDR);
    uint2* ranges = ws_ptr<uint2>(ws, p, OFF_RANGES);
    int launches = 0;
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)p.n_tiles, st);
    if (total == 0 || p.capacity == 0) {
        // no instances: every tile is empty, the schedule is still needed
        tile_order_kernel<<<1, 1024, 0, st>>>(ranges, p.n_tiles, ws_ptr<uint32_t>(ws, p, OFF_ORDER));
        return launches + 1;
    }
    uint32_t* touched = ws_ptr<uint32_t>(ws, p, OFF_TOUCH);
    uint32_t* offs = ws_ptr<uint32_t>(ws, p, OFF_OFFS);
    uint32_t* scan_tmp = ws_ptr<uint32_t>(ws, p, OFF_SCAN);
    launches += scan_u32(touched, total, scan_tmp, offs, nullptr, st);
    unsigned long long* keys[2] = {ws_ptr<unsigned long long>(ws, p, OFF_KEYS0),
                                   ws_ptr<unsigned long long>(ws, p, OFF_KEYS1)};
    uint32_t* vals[2] = {ws_ptr<uint32_t>(ws, p, OFF_VALS0), ws_ptr<uint32_t>(ws, p, OFF_VALS1)};
    {
        const int64_t blocks = (total + 255) / 256;
        const int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
        emit_kernel<<<grid, 256, 0, st>>>(ws_ptr<CamTable>(ws, p, OFF_CAM), p.n, p.n_cams,
                                          p.cfg.tile_w, p.cfg.tile_h, p.capacity, ws_ptr<uint2>(ws, p, OFF_RECT), touched,
                                          offs, ws_ptr<uint32_t>(ws, p, OFF_ZBITS),
                                          ws_ptr<float>(ws, p, OFF_CULL), hdr, keys[0], vals[0]);
        ++launches;
    }
    const int nb = (int)((p.capacity + SORT_ITEMS - 1) / SORT_ITEMS);
    uint32_t* hist = ws_ptr<uint32_t>(ws, p, OFF_HIST);
    for (int pass = 0; pass < p.sort_passes; ++pass) {
        const int src = pass & 1, dst = src ^ 1;
        radix_hist_kernel<<<nb, 256, 0, st>>>(keys[src], hdr, 8 * pass, 255u, nb, hist);
        launches += 1 + scan_u32(hist, (int64_t)nb * 256, scan_tmp, hist, nullptr, st);
        radix_scatter_kernel<<<nb, 256, 0, st>>>(keys[src], vals[src], keys[dst], vals[dst], hist,
                                                 hdr, 8 * pass, 255u, nb);
        ++launches;
    }
    const int fin = sorted_buffer(p);
    {
        const int64_t blocks = (p.capacity + 255) / 256;
        const int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
        ranges_kernel<<<grid, 256, 0, st>>>(keys[fin], hdr, ranges);
        ++launches;
    }
    tile_order_kernel<<<1, 1024, 0, st>>>(ranges, p.n_tiles, ws_ptr<uint32_t>(ws, p, OFF_ORDER));
    ++launches;
    return launches;
}

}  // namespace unigs
