// peak.cu -- FP32 issue-rate measurement behind vafr_measure_fp32_peak: the
// denominator of the traversal kernels' ALU roofline, measured on the device
// that runs them rather than derived from lane counts and a nominal clock.
#include "vafr_internal.cuh"

namespace vafr {
namespace {

constexpr int kChains = 8;    // independent FMA chains per thread (hides the pipe latency)
constexpr int kUnroll = 16;   // FMA rounds per loop trip

// Every thread runs kChains independent chains x = x a + b (scalar FFMA, or
// paired FFMA2 on float2) for iters x kUnroll rounds.  |a| < 1 keeps the
// values bounded; the sum is stored only when it equals a value it never
// takes, which keeps the chains alive without a memory stream.
template <bool PAIRED>
__global__ void __launch_bounds__(256) k_fma_peak(float a, float b, int iters, float* sink) {
    if (PAIRED) {
        float2 x[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = make_float2(threadIdx.x * 1e-7f + i, blockIdx.x * 1e-7f - i);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
        if (s == -1.2345e30f) sink[blockIdx.x] = s;
    } else {
        float x[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 1e-7f + i;
#pragma unroll 1
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i];
        if (s == -1.2345e30f) sink[blockIdx.x] = s;
    }
}

template <bool PAIRED>
cudaError_t time_one(int grid, int iters, float* sink, cudaStream_t s, double* fma_per_s) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    float best = INFINITY;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_peak<PAIRED><<<grid, 256, 0, s>>>(0.9999999f, 1e-7f, iters, sink);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;   // launch 0 warms up
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)grid * 256.0 * iters * kUnroll * kChains * (PAIRED ? 2.0 : 1.0);
    *fma_per_s = e == cudaSuccess && best > 0.0f ? fmas / (best * 1e-3) : 0.0;
    count_launch(4);
    return e;
}

}  // namespace

cudaError_t measure_fp32_peak(int num_sms, float* sink, cudaStream_t s, double* ffma, double* ffma2) {
    const int grid = num_sms * 8;    // 2,048 threads per SM
    cudaError_t e = time_one<false>(grid, 3000, sink, s, ffma);
    if (e == cudaSuccess) e = time_one<true>(grid, 3000, sink, s, ffma2);
    return e;
}

}  // namespace vafr
