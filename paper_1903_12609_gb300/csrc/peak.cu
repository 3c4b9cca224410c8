// Measured FMA rates of the GPU (fil_fma_peak): the measured counterpart of
// the derived FP32 and FP64 peaks (SMs x lanes x 2 flops x clock) against
// which the pair kernels' roofline fractions are reported.
//
// Every thread runs kPeakChains independent chains x <- x b + c (b < 1, so x
// converges to c / (1 - b) and stays a normal number), packed FP32x2 FMAs or
// FP64 FMAs, with enough resident warps per SM to hide the FMA latency. Thread
// 0 of CTA 0 reads clock64 and the global nanosecond timer around its loop,
// which gives the SM clock during the run.
#include <cuda_runtime.h>

#include "fil_internal.cuh"

namespace fil {
namespace {

constexpr int kPeakChains = 8;     // independent chains per thread
constexpr int kPeakInner = 16;     // FMAs per chain per outer iteration
constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 8;  // 2048 threads per SM

__device__ unsigned long long g_peak_clk[2];   // cycles, nanoseconds of CTA 0's loop
__device__ double g_peak_sink;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kPeakThreads) fma_peak32_kernel(int iters) {
    float2 x[kPeakChains];
    const float2 b = make_float2(0.9990f, 0.9993f), c = make_float2(1.0e-3f, 0.7e-3f);
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = make_float2(1e-3f * threadIdx.x, (float)j);
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    long long c0 = 0;
    unsigned long long t0 = 0;
    if (timer) { c0 = clock64(); t0 = global_ns(); }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < kPeakInner; ++r)
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) x[j] = __ffma2_rn(x[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += x[j].x + x[j].y;
    if (s == -1.f) g_peak_sink = s;   // never true: keeps the chains live
    if (timer) {
        g_peak_clk[0] = (unsigned long long)(clock64() - c0);
        g_peak_clk[1] = global_ns() - t0;
    }
}

__global__ void __launch_bounds__(kPeakThreads) fma_peak64_kernel(int iters) {
    double x[kPeakChains];
    const double b = 0.9990, c = 1.0e-3;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = 1e-3 * threadIdx.x + j;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    long long c0 = 0;
    unsigned long long t0 = 0;
    if (timer) { c0 = clock64(); t0 = global_ns(); }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < kPeakInner; ++r)
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) x[j] = fma(x[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += x[j];
    if (s == -1.0) g_peak_sink = s;
    if (timer) {
        g_peak_clk[0] = (unsigned long long)(clock64() - c0);
        g_peak_clk[1] = global_ns() - t0;
    }
}

}  // namespace
}  // namespace fil

extern "C" fil_status fil_fma_peak(int32_t fp64, double *flops_per_s, double *sm_mhz) {
    using namespace fil;
    if (fp64 != 0 && fp64 != 1) return FIL_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FIL_ECUDA;
    const int grid = sms * kPeakCtasPerSm;
    // ~20 ms per launch at the nominal rates (FP32x2: 256 lanes x 2 flops per
    // SM clock; FP64: 2 lanes x 2 flops)
    const int iters = fp64 ? 320 : 10000;
    const double flops = (double)grid * kPeakThreads * iters * kPeakInner * kPeakChains *
                         (fp64 ? 2.0 : 4.0);
    auto launch = [&]() {
        if (fp64) fma_peak64_kernel<<<grid, kPeakThreads>>>(iters);
        else fma_peak32_kernel<<<grid, kPeakThreads>>>(iters);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FIL_ECUDA;
    }
    constexpr int kReps = 5;
    launch();   // warm-up (clocks ramp, code paged in)
    cudaEventRecord(e0, 0);
    for (int r = 0; r < kReps; ++r) launch();
    cudaEventRecord(e1, 0);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long clk[2] = {0, 0};
    if (err == cudaSuccess) err = cudaMemcpyFromSymbol(clk, g_peak_clk, sizeof(clk));
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || !(ms > 0.f)) return FIL_ECUDA;
    if (flops_per_s) *flops_per_s = kReps * flops / (ms * 1e-3);
    if (sm_mhz) *sm_mhz = clk[1] ? 1e3 * (double)clk[0] / (double)clk[1] : 0.0;
    return FIL_OK;
}
