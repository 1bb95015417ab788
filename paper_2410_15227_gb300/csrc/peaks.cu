// Measured arithmetic peaks of the device (em_measure_peaks): the rates that
// the roofline of the ALU-bound mapping kernels is reported against.  Each
// kernel runs independent dependency chains, enough per thread and threads
// per SM that the pipe, not latency, limits it, over a grid of
// (SMs x blocks per SM), and is timed with CUDA events over a region of tens
// of milliseconds.  The results are written to out[] only; nothing is kept.
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;   // independent chains per thread

// FP32 fused multiply-add: 2 flops each.  The multiplier and addend keep the
// chains bounded (|x| stays below 2) so that no value becomes special.
__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(int iters, float a, float b, float *out)
{
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 0.001f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == 12345.678f) out[0] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(int iters, double a, double b, double *out)
{
    double x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 0.001 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;
}

// One special-function (XU) operation per step: the approximate reciprocal
// square root, whose chains x <- rsqrt(x) + b stay near a fixed point.
__global__ void __launch_bounds__(PK_THREADS) k_peak_xu(int iters, float b, float *out)
{
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1.0f + 0.001f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = rsqrtf(x[c]) + b;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == 12345.678f) out[0] = s;
}

// Milliseconds of one launch, the median of 3 after a warm-up launch.
template <class F>
int time_launch(cudaStream_t st, F launch, float *ms)
{
    cudaEvent_t e0, e1;
    EM_CUDA(cudaEventCreate(&e0));
    EM_CUDA(cudaEventCreate(&e1));
    launch();
    float t[3];
    int rc = EM_OK;
    for (int r = 0; r < 3 && rc == EM_OK; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess) {
            em_set_error("em_measure_peaks: timing failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = EM_ECUDA;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != EM_OK) return rc;
    const float lo = fminf(t[0], fminf(t[1], t[2])), hi = fmaxf(t[0], fmaxf(t[1], t[2]));
    *ms = t[0] + t[1] + t[2] - lo - hi;
    return EM_OK;
}

}  // namespace

EM_EXPORT int em_measure_peaks(em_ctx *ctx, double *h_out)
{
    EM_CHECK_ARG(ctx && h_out);
    cudaStream_t st = ctx->stream;
    DevArena tmp(st, true);
    float *sink_f;
    double *sink_d;
    EM_TRY(tmp.alloc(&sink_f, 1));
    EM_TRY(tmp.alloc(&sink_d, 1));
    int per_sm = 0;
    EM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_ffma, PK_THREADS, 0));
    const int grid = ctx->nsm * (per_sm > 0 ? per_sm : 1);
    const double threads = (double)grid * PK_THREADS;
    // iterations sized for tens of milliseconds at the nominal rates
    const int it32 = 20000, it64 = 300, itxu = 2500;
    float ms;
    EM_TRY(time_launch(st, [&] { k_peak_ffma<<<grid, PK_THREADS, 0, st>>>(it32, 0.999f, 0.001f, sink_f); }, &ms));
    ctx->launches += 3;   // four launches per measurement
    EM_LAUNCHED(ctx);
    h_out[0] = threads * it32 * 16.0 * PK_CHAINS * 2.0 / (ms * 1e-3) / 1e12;
    EM_TRY(time_launch(st, [&] { k_peak_dfma<<<grid, PK_THREADS, 0, st>>>(it64, 0.999, 0.001, sink_d); }, &ms));
    ctx->launches += 3;
    EM_LAUNCHED(ctx);
    h_out[1] = threads * it64 * 16.0 * PK_CHAINS * 2.0 / (ms * 1e-3) / 1e12;
    EM_TRY(time_launch(st, [&] { k_peak_xu<<<grid, PK_THREADS, 0, st>>>(itxu, 0.5f, sink_f); }, &ms));
    ctx->launches += 3;
    EM_LAUNCHED(ctx);
    h_out[2] = threads * itxu * 16.0 * PK_CHAINS / (ms * 1e-3) / 1e12;
    int clock_khz = 0;
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, ctx->device);
    h_out[3] = (double)ctx->nsm;
    h_out[4] = clock_khz * 1e-3;
    return EM_OK;
}
