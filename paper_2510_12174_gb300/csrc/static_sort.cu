// unigs_sort_pairs_static: the library's stable radix sort of (key, value)
// pairs, with its scratch memory in a file-scope device array instead of a
// caller-allocated workspace.
//
// It exists for callers that cannot allocate device memory at the point of
// the call: code running under a fixed memory budget fixed at start-up, a
// plugin host that owns all allocations, or a real-time loop where a
// cudaMalloc (which may synchronise the device) is not allowed.  They pass
// only their inputs and outputs.
//
// The scratch (one key/value ping-pong buffer, the per-block digit histograms,
// the scan partials and a status block) lives in g_sort_scratch, about 12.5 MB
// that every GPU which loads the library keeps until the process exits.  In
// host code g_sort_scratch is only a host-side stand-in for the symbol, not a
// device address: the first call on each device (with that device current)
// looks its device address up with cudaGetSymbolAddress and caches it, so that
// first call should come before any stream capture.  All calls share the one
// array: calls that overlap on the GPU (different streams, or several host
// threads) race on it.
#include <mutex>

#include "launch.h"

namespace unigs {
namespace {

constexpr int64_t STATIC_MAX_PAIRS = UNIGS_STATIC_SORT_MAX_PAIRS;
constexpr int64_t STATIC_MAX_BLOCKS = (STATIC_MAX_PAIRS + SORT_ITEMS - 1) / SORT_ITEMS;
constexpr int64_t STATIC_MAX_PARTIALS = (256 * STATIC_MAX_BLOCKS + SCAN_ITEMS - 1) / SCAN_ITEMS;

struct StaticSortScratch {
    WsHeader hdr;                              // status + pair count read by the kernels
    unsigned long long keys[STATIC_MAX_PAIRS]; // ping-pong partner of the output
    uint32_t vals[STATIC_MAX_PAIRS];
    uint32_t hist[256 * STATIC_MAX_BLOCKS];    // per-block digit counts, then their scan
    uint32_t partial[STATIC_MAX_PARTIALS + 16];
};

__device__ __align__(256) unsigned char g_sort_scratch[sizeof(StaticSortScratch)];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_dev[MAX_DEVICES] = {};

// Device address of g_sort_scratch on the current device (cached per device).
cudaError_t scratch_on_current_device(StaticSortScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = static_cast<StaticSortScratch*>(g_scratch_dev[dev]);
    return cudaSuccess;
}

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// Every call starts from a clean status block holding its own pair count.
__global__ void static_sort_init_kernel(StaticSortScratch* s, uint32_t n) {
    s->hdr.status = 0;
    s->hdr.n_instances = n;
    s->hdr.need = n;
}

}  // namespace
}  // namespace unigs

using namespace unigs;

extern "C" unigs_status unigs_sort_pairs_static(const unsigned long long* keys_in,
                                                const uint32_t* vals_in, int64_t n,
                                                int32_t key_bits, unsigned long long* keys_out,
                                                uint32_t* vals_out, unigs_stream stream) {
    if (n < 0 || n > STATIC_MAX_PAIRS || key_bits < 1 || key_bits > 64)
        return UNIGS_ERR_INVALID_ARG;
    if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out)) return UNIGS_ERR_INVALID_ARG;
    if (n > 0) {
        // an output may share no byte with an input or with the other output
        // (the passes ping-pong between the outputs and the static scratch)
        const size_t kb = sizeof(unsigned long long) * (size_t)n, vb = sizeof(uint32_t) * (size_t)n;
        if (overlap(keys_out, kb, keys_in, kb) || overlap(keys_out, kb, vals_in, vb) ||
            overlap(keys_out, kb, vals_out, vb) || overlap(vals_out, vb, keys_in, kb) ||
            overlap(vals_out, vb, vals_in, vb))
            return UNIGS_ERR_INVALID_ARG;
    }
    StaticSortScratch* s = nullptr;
    if (scratch_on_current_device(&s) != cudaSuccess) return UNIGS_ERR_CUDA;
    if (n == 0) return UNIGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    static_sort_init_kernel<<<1, 1, 0, st>>>(s, (uint32_t)n);
    const int passes = (key_bits + 7) / 8;
    const int nb = (int)((n + SORT_ITEMS - 1) / SORT_ITEMS);
    // the last pass sorts by the key_bits - 8 (passes - 1) bits that remain,
    // so key bits at and above key_bits never decide the order
    const int last_bits = key_bits - 8 * (passes - 1);
    // pass p writes the output when (passes - 1 - p) is even, else the
    // scratch buffer, so the last pass lands in the output and consecutive
    // passes never read and write the same buffer.
    const unsigned long long* kin = keys_in;
    const uint32_t* vin = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) & 1) == 0;
        unsigned long long* kout = to_out ? keys_out : s->keys;
        uint32_t* vout = to_out ? vals_out : s->vals;
        const uint32_t dmask = p == passes - 1 ? (1u << last_bits) - 1u : 255u;
        radix_pass(kin, vin, kout, vout, s->hist, s->partial, &s->hdr, 8 * p, dmask, nb, st);
        kin = kout;
        vin = vout;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? UNIGS_OK : UNIGS_ERR_CUDA;
}
