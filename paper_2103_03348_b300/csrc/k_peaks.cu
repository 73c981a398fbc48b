// ALU throughput microbenchmarks, the denominators of the FP32 roofline:
// packed FP32 FMA (f32x2, the row and column passes' instruction), the MUFU
// exp2 and FP64 FMA.  Each thread runs independent dependency chains long
// enough to hide latency; the result is folded into a sink so no work can be
// removed.  The caller times the launch with CUDA events on its stream.
#include "hawkes_internal.cuh"

namespace hk {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_UNROLL = 8;  // iterations per loop trip, so loop control is negligible

__global__ void __launch_bounds__(PEAK_THREADS) peak_ffma2_kernel(int iters, float seed, float *sink) {
    float2 acc[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = make_float2(seed + c, seed - c);
    const float2 m = make_float2(0.9999f, 1.0001f), a = make_float2(1.0e-7f, -1.0e-7f);
    for (int i = 0; i < iters; i += PEAK_UNROLL) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = fma2(acc[c], m, a);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += acc[c].x + acc[c].y;
    if (s == 12345.678f) sink[0] = s;  // practically never true; keeps the chains live
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_ex2_kernel(int iters, float seed, float *sink) {
    float v[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) v[c] = seed * (c + 1);
    for (int i = 0; i < iters; i += PEAK_UNROLL) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) v[c] = ex2_ftz(v[c]) - 1.0f;  // stays in [-1, 1]
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += v[c];
    if (s == 12345.678f) sink[0] = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_dfma_kernel(int iters, double seed, float *sink) {
    double acc[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = seed + c;
    for (int i = 0; i < iters; i += PEAK_UNROLL) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = fma(acc[c], 0.9999999, 1.0e-9);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += acc[c];
    if (s == 12345.678) sink[0] = (float)s;
}

}  // namespace hk

extern "C" {

int64_t hawkes_peak_ops(int which, int64_t blocks, int iters) {
    if (which < 0 || which > 2 || blocks < 1 || iters < 1 || iters % hk::PEAK_UNROLL) return 0;
    const int64_t lanes = which == 0 ? 2 : 1;  // an f32x2 FMA is two lane operations
    return blocks * hk::PEAK_THREADS * (int64_t)iters * hk::PEAK_CHAINS * lanes;
}

int hawkes_peak_launch(int which, int64_t blocks, int iters, float *sink, void *stream) {
    if (which < 0 || which > 2 || blocks < 1 || blocks > 0x7fffffff || iters < 1 || iters % hk::PEAK_UNROLL || !sink)
        return HAWKES_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = (unsigned)blocks;
    if (which == 0) hk::peak_ffma2_kernel<<<g, hk::PEAK_THREADS, 0, s>>>(iters, 1.0f, sink);
    else if (which == 1) hk::peak_ex2_kernel<<<g, hk::PEAK_THREADS, 0, s>>>(iters, 0.25f, sink);
    else hk::peak_dfma_kernel<<<g, hk::PEAK_THREADS, 0, s>>>(iters, 1.0, sink);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

}  // extern "C"
