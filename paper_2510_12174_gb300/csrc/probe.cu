// FP32 FMA throughput probe (a measurement utility; the paper has no
// counterpart).  The composite kernels are bound by FP32 arithmetic and
// issue, so their roofline is taken against the FMA rate this GPU actually
// sustains, measured here rather than derived from unit counts and clocks.
//
// Every thread runs 8 independent FMA chains (enough to cover the FMA
// latency with the 64 resident warps per SM of this launch shape), either as
// scalar fmaf or as packed float32 pairs (__ffma2_rn, two FMAs per
// instruction).  The grid is 8 CTAs of 256 threads per SM.  The results are
// folded into one store per thread so that no chain can be removed.
#include "launch.h"

namespace unigs {
namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 8;

__global__ void __launch_bounds__(PROBE_THREADS)
    fma_probe_kernel(float* __restrict__ sink, int iters, float a, float b) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS)
    fma2_probe_kernel(float* __restrict__ sink, int iters, float a, float b) {
    float2 x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k)
        x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x - k) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k].x + x[k].y;
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace unigs

using namespace unigs;

extern "C" int64_t unigs_probe_fma_sink_floats(void) {
    return (int64_t)sm_count() * PROBE_CTAS_PER_SM * PROBE_THREADS;
}

extern "C" unigs_status unigs_probe_fma(float* sink, int32_t iters, int32_t packed,
                                        int64_t* flops_out, unigs_stream stream) {
    if (!sink || iters < 1 || (packed != 0 && packed != 1)) return UNIGS_ERR_INVALID_ARG;
    const int grid = sm_count() * PROBE_CTAS_PER_SM;
    // a and b keep every chain finite and away from subnormals
    const float a = 0.999999f, b = 1e-6f;
    if (packed)
        fma2_probe_kernel<<<grid, PROBE_THREADS, 0, (cudaStream_t)stream>>>(sink, iters, a, b);
    else
        fma_probe_kernel<<<grid, PROBE_THREADS, 0, (cudaStream_t)stream>>>(sink, iters, a, b);
    if (flops_out)
        *flops_out = (int64_t)grid * PROBE_THREADS * (int64_t)iters * 16 * PROBE_CHAINS *
                     (packed ? 4 : 2);
    return cudaGetLastError() == cudaSuccess ? UNIGS_OK : UNIGS_ERR_CUDA;
}
