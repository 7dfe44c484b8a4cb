// k_peak.cu -- FP32 FMA throughput microbenchmark, the denominator of the
// ALU roofline the benchmark reports for the FP32 transforms (no
// counterpart in the paper).  Each thread runs 8 independent chains of
// packed f32x2 FMAs; the CTAs fill every SM several times over.
#include <cuda_runtime.h>

#include "ctx.h"
#include "fft_block.cuh"
#include "spec.h"

namespace spec {

constexpr int kPeakIters = 4096;
constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(256) k_fp32_peak(float* sink, float seed) {
    float2 acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = make_float2(seed + c, seed - c + threadIdx.x);
    const float2 a = make_float2(0.999999f, 1.000001f), b = make_float2(1e-7f, -1e-7f);
#pragma unroll 4
    for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) acc[c] = fma2(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += acc[c].x + acc[c].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;          // keeps the chains live
}

}  // namespace spec

extern "C" spec_status spec_measure_fp32_peak(spec_ctx* c, double* tflops, void* stream) {
    if (!c || !tflops) return SPEC_EINVAL;
    *tflops = 0.0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = std::max(1, c->sms) * 8;
    const int threads = 256;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, threads * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; e == cudaSuccess && rep < 6; ++rep) {
        e = cudaEventRecord(e0, st);
        spec::k_fp32_peak<<<blocks, threads, 0, st>>>(sink, 1.0f + rep);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) {
            const double flops = 2.0 * 2.0 * spec::kPeakChains * (double)spec::kPeakIters * blocks * threads;
            best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaSetDevice(dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return spec::ctx_cuda_fail(c, e, "FP32 peak measurement");
    }
    *tflops = best;
    return SPEC_OK;
}
