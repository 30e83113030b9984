// reed_peaks.cu -- throughput microbenchmarks for the roofline of the track
// stepper: FP32 FMA, FP64 FMA, the SFU's ex2 and rsqrt, and 128-bit shared-
// memory loads, each as many independent streams per thread so that issue
// (not latency) is the limit.  The stepper is bound by these units, not by
// HBM or the tensor cores.
#include <cuda_runtime.h>

#include <cstring>

#include "reed.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_kernel(int iters, T a, T b, T* __restrict__ sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;   // never true; keeps the chains alive
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) sfu_kernel(int iters, float* __restrict__ sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = OP == 0 ? ex2_approx(x[c]) : rsqrt_approx(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) lds_kernel(int iters, float* __restrict__ sink)
{
    __shared__ float4 buf[kThreads * 2];
    for (int i = threadIdx.x; i < kThreads * 2; i += blockDim.x) buf[i] = make_float4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    float4 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    // consecutive lanes read consecutive 16-byte words: no bank conflicts
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 v = buf[(idx + c * 32) & (kThreads * 2 - 1)];
            acc[c].x += v.x;
            acc[c].y += v.y;
            acc[c].z += v.z;
            acc[c].w += v.w;
        }
        idx = (idx + 128) & (kThreads * 2 - 1);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) s += acc[c].x + acc[c].y + acc[c].z + acc[c].w;
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

__global__ void clock_kernel(long long cycles, long long* __restrict__ out)
{
    const long long t0 = clock64();
    while (clock64() - t0 < cycles) {
    }
    if (threadIdx.x == 0) out[blockIdx.x] = clock64() - t0;
}

}  // namespace

extern "C" int reed_peaks(reed_peaks_t* out)
{
    if (!out) return REED_E_ARG;
    std::memset(out, 0, sizeof(*out));
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return REED_E_CUDA;
    void* sink = nullptr;
    if (cudaMalloc(&sink, 1 << 16) != cudaSuccess) return REED_E_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = 4 * sms;   // 4 CTAs x 512 threads per SM
    const double threads = (double)grid * kThreads;
    auto timed = [&](auto launch) -> double {
        launch();   // warm-up
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3;
    };
    const int it32 = 1 << 15, it64 = 1 << 11, itsfu = 1 << 13, itlds = 1 << 13;
    double s;
    s = timed([&] { fma_kernel<float><<<grid, kThreads>>>(it32, 1.0000001f, 1e-7f, (float*)sink); });
    out->fp32_tflops = threads * it32 * kChains * 2.0 / s * 1e-12;
    s = timed([&] { fma_kernel<double><<<grid, kThreads>>>(it64, 1.0000001, 1e-7, (double*)sink); });
    out->fp64_tflops = threads * it64 * kChains * 2.0 / s * 1e-12;
    s = timed([&] { sfu_kernel<0><<<grid, kThreads>>>(itsfu, (float*)sink); });
    out->ex2_gops = threads * itsfu * kChains / s * 1e-9;
    s = timed([&] { sfu_kernel<1><<<grid, kThreads>>>(itsfu, (float*)sink); });
    out->rsqrt_gops = threads * itsfu * kChains / s * 1e-9;
    s = timed([&] { lds_kernel<<<grid, kThreads>>>(itlds, (float*)sink); });
    out->smem_tbs = threads * itlds * 4 * 16.0 / s * 1e-12;
    // SM clock under load: cycles counted by one CTA per SM over a known time
    const long long cyc = 200000000LL;
    s = timed([&] { clock_kernel<<<sms, 32>>>(cyc, (long long*)sink); });
    out->sm_mhz = (double)cyc / s * 1e-6;
    out->sms = sms;
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return err == cudaSuccess ? REED_OK : REED_E_CUDA;
}
