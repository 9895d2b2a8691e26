// Throughput calibration of the units the hot path is bound by: FP32 fused
// multiply-add, FP64 fused multiply-add, the special-function unit
// (single-instruction approximate rsqrt and sin, the forms the mixed
// quadrature uses) and a device-memory copy.  Each kernel keeps many
// independent dependency chains per thread, so that issue and pipe
// throughput, not latency, set its time; every chain's result is folded
// into one value that is written only when it is impossible, so the work
// cannot be removed by the compiler.  The rates are the roofline
// denominators of the benchmark (bem_measure_peaks).
#include <algorithm>
#include <cstring>

#include "../../include/bem.h"
#include "bem_internal.h"

namespace bem {
namespace {

constexpr int kCalThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kCalThreads) k_cal_ffma(float *sink, int iters, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = (float)(threadIdx.x + q);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int q = 0; q < kChains; ++q) a[q] = fmaf(a[q], b, c);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kCalThreads) k_cal_dfma(double *sink, int iters, double b, double c)
{
    double a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = (double)(threadIdx.x + q);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == -1.2345) sink[blockIdx.x] = (double)s;
}

// MUFU: y <- rsqrt(y) (or sin(y)) on independent chains; no other work in
// the loop body, so the special-function pipe alone limits it
template <int FN>
__global__ void __launch_bounds__(kCalThreads) k_cal_mufu(float *sink, int iters)
{
    float a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = 1.5f + 0.01f * (float)(threadIdx.x + q);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < kChains; ++q) {
                float r;
                if (FN == 0) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[q]));
                else asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[q]));
                a[q] = r;
            }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void k_cal_copy(const float4 *__restrict__ src, float4 *__restrict__ dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" int bem_measure_peaks(bem_peaks *out, void *cuda_stream)
{
    if (!out) {
        set_last_error("out is null");
        return BEM_E_ARG;
    }
    std::memset(out, 0, sizeof(*out));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, clk_khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return BEM_E_CUDA;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cal_ffma, kCalThreads, 0);
    const int grid = sms * std::max(per_sm, 1);
    const int64_t threads = (int64_t)grid * kCalThreads;
    // copy: 2 x 1 GiB (read + write)
    const int64_t copy_bytes = int64_t(1) << 30;
    void *buf = nullptr, *src = nullptr, *dst = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&buf, 2 * copy_bytes + 4096);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 2 * copy_bytes + 4096, st);
    src = buf;
    dst = (char *)buf + copy_bytes;
    float *sinkf = (float *)((char *)buf + 2 * copy_bytes);
    double *sinkd = (double *)sinkf;
    // best of 3 timed launches after one warm-up; returns ms
    auto time_it = [&](auto launch) -> float {
        float best = 1e30f;
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
            cudaEventRecord(a, st);
            launch();
            cudaEventRecord(b, st);
            e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (r > 0) best = std::min(best, ms);
        }
        return best;
    };
    const int it_f = 2048, it_d = 64, it_m = 512;
    float ms_f = time_it([&] { k_cal_ffma<<<grid, kCalThreads, 0, st>>>(sinkf, it_f, 0.999f, 1e-3f); });
    float ms_d = time_it([&] { k_cal_dfma<<<grid, kCalThreads, 0, st>>>(sinkd, it_d, 0.999, 1e-3); });
    float ms_r = time_it([&] { k_cal_mufu<0><<<grid, kCalThreads, 0, st>>>(sinkf, it_m); });
    float ms_s = time_it([&] { k_cal_mufu<1><<<grid, kCalThreads, 0, st>>>(sinkf, it_m); });
    const int64_t n4 = copy_bytes / 16;
    float ms_c = time_it([&] {
        k_cal_copy<<<sms * 8, 512, 0, st>>>((const float4 *)src, (float4 *)dst, n4);
    });
    count_launches(20);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (buf) cudaFree(buf);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return BEM_E_CUDA;
    }
    out->fp32_fma_per_s = (double)threads * it_f * 16 * kChains / (ms_f * 1e-3);
    out->fp64_fma_per_s = (double)threads * it_d * 4 * kChains / (ms_d * 1e-3);
    out->mufu_rsqrt_per_s = (double)threads * it_m * 4 * kChains / (ms_r * 1e-3);
    out->mufu_sin_per_s = (double)threads * it_m * 4 * kChains / (ms_s * 1e-3);
    out->copy_bytes_per_s = 2.0 * (double)copy_bytes / (ms_c * 1e-3);
    out->sm_count = sms;
    out->clock_mhz_nominal = clk_khz / 1000.0;
    out->ms[0] = ms_f;
    out->ms[1] = ms_d;
    out->ms[2] = ms_r;
    out->ms[3] = ms_s;
    out->ms[4] = ms_c;
    return BEM_OK;
}
