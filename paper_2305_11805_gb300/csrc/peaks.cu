// Throughput of the two arithmetic units that bound the descriptor family: the FP32 FMA
// pipe (the outer products, polynomial and geometry arithmetic of every pair term) and the
// multi-function unit's ex2 (the Gaussians and zeta powers).  The angular kernels are not
// HBM-bound (hundreds of FP32 operations per byte), so their roofline is this unit's peak;
// measuring it on the GPU at hand, with the clocks of the moment, gives the denominator of
// their efficiency instead of a figure derived from unit counts and the maximum clock.
//
// Each kernel runs independent dependency chains per thread (enough in flight to hide the
// pipe latency at full occupancy) on every SM, timed with CUDA events on the caller's
// stream; the best of several launches is reported.
#include <stdio.h>

#include "common.cuh"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;     // 2048 resident threads per SM
constexpr int kChains = 8;              // independent chains per thread
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float* out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) out[blockIdx.x] = s;   // keeps the chains live; practically never taken
}

// the same chains with packed two-wide FP32 FMAs (one instruction, two FMAs per lane)
__global__ void __launch_bounds__(kPeakThreads) k_fma2_peak(float* out, int iters, float a, float b)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) x[k] = make_float2(1e-3f * (float)threadIdx.x + (float)k, (float)k - 1.f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) s += x[k].x + x[k].y;
    if (s == 1234.5f) out[blockIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 2^(-x) stays in (0, 1): one MUFU operation per step (the negation folds into it)
__global__ void __launch_bounds__(kPeakThreads) k_ex2_peak(float* out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-4f * (float)threadIdx.x + 0.1f * (float)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = ex2_approx(-x[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" panna_status panna_measure_alu_peaks2(double* fp32_tflops, double* fp32x2_tflops, double* ex2_gops,
                                                 panna_stream_t stream);

extern "C" panna_status panna_measure_alu_peaks(double* fp32_tflops, double* ex2_gops, panna_stream_t stream)
{
    double packed = 0.0;
    return panna_measure_alu_peaks2(fp32_tflops, &packed, ex2_gops, stream);
}

extern "C" panna_status panna_measure_alu_peaks2(double* fp32_tflops, double* fp32x2_tflops, double* ex2_gops,
                                                 panna_stream_t stream)
{
    if (!fp32_tflops || !fp32x2_tflops || !ex2_gops) {
        panna::set_last_error_message("null argument");
        return PANNA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    float* sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&sink, sizeof(float) * (size_t)n_sm * kPeakBlocksPerSm, s);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const unsigned blocks = (unsigned)(n_sm * kPeakBlocksPerSm);
    const double threads = (double)blocks * kPeakThreads;
    const int fma_iters = 20000, ex2_iters = 2000;
    double best_fma = 0.0, best_ex2 = 0.0, best_fma2 = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        float ms = 0.f;
        e = cudaEventRecord(t0, s);
        if (e == cudaSuccess) {
            k_fma_peak<<<blocks, kPeakThreads, 0, s>>>(sink, fma_iters, 0.9999999f, 1e-7f);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) {   // the first launch is a warm-up
            const double fl = 2.0 * threads * fma_iters * kUnroll * kChains;
            if (fl / (ms * 1e-3) / 1e12 > best_fma) best_fma = fl / (ms * 1e-3) / 1e12;
        }
        if (e == cudaSuccess) e = cudaEventRecord(t0, s);
        if (e == cudaSuccess) {
            k_fma2_peak<<<blocks, kPeakThreads, 0, s>>>(sink, fma_iters, 0.9999999f, 1e-7f);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) {
            const double fl = 2.0 * threads * fma_iters * kUnroll * kChains;
            if (fl / (ms * 1e-3) / 1e12 > best_fma2) best_fma2 = fl / (ms * 1e-3) / 1e12;
        }
        if (e == cudaSuccess) e = cudaEventRecord(t0, s);
        if (e == cudaSuccess) {
            k_ex2_peak<<<blocks, kPeakThreads, 0, s>>>(sink, ex2_iters);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) {
            const double ops = threads * ex2_iters * kUnroll * kChains;
            if (ops / (ms * 1e-3) / 1e9 > best_ex2) best_ex2 = ops / (ms * 1e-3) / 1e9;
        }
    }
    if (sink) {
        cudaError_t e2 = cudaFreeAsync(sink, s);
        if (e == cudaSuccess) e = e2;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "peak measurement: %s", cudaGetErrorString(e));
        panna::set_last_error_message(msg);
        return PANNA_ERR_CUDA;
    }
    *fp32_tflops = best_fma;
    *fp32x2_tflops = best_fma2;
    *ex2_gops = best_ex2;
    return PANNA_OK;
}
