// Throughput probes of the three units that bound one scoring evaluation:
// the FP32 pipe (fused multiply-adds, scalar and two-wide), the special-
// function unit (ex2 for the pair terms' two exponentials, rsqrt standing in
// for their rsqrt and reciprocal) and random 16-byte gathers from an L2-resident buffer about the
// size of a receptor's packed maps (64^3 points x 16 bytes = 4 MiB; the
// probe uses 8 MiB).  Each probe is one launch of every SM's worth of warps,
// timed with CUDA events on the context's stream after one untimed launch.

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "adg_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;  // 64 warps per SM: every scheduler has warps to pick from
constexpr int kChains = 8;       // independent dependency chains per thread
constexpr int kFmaIters = 16384;
constexpr int kEx2Iters = 4096;
constexpr int kGatherIters = 1024;
constexpr int kGatherLoads = 8;  // loads in flight per thread and iteration
constexpr uint32_t kGatherElems = 1u << 19;  // float4 elements: 8 MiB

// a result the compiler cannot prove unused; the comparison is never true for
// the bounded values these chains produce
__device__ __forceinline__ void keep(float s, float* sink)
{
    if (s == 1234567.f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_fma(float seed, int iters, float* sink)
{
    float a[2 * kChains];
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) a[i] = seed + 0.01f * i + 1e-5f * threadIdx.x;
    const float m = 0.99990f, c = 1e-4f;
#pragma unroll 4
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 2 * kChains; ++i) a[i] = fmaf(a[i], m, c);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) s += a[i];
    keep(s, sink);
}

__global__ void __launch_bounds__(kThreads) k_peak_fma2(float seed, int iters, float* sink)
{
    float2 a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = make_float2(seed + 0.01f * i + 1e-5f * threadIdx.x, seed - 0.01f * i);
    const float2 m = make_float2(0.99990f, 0.99990f), c = make_float2(1e-4f, 1e-4f);
#pragma unroll 4
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], m, c);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
    keep(s, sink);
}

__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 2^-x stays in [0.5, 1] for x in [0, 1]
__global__ void __launch_bounds__(kThreads) k_peak_ex2(float seed, int iters, float* sink)
{
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = seed * (i + 1) * 0.1f + 1e-6f * threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = ex2_ftz(-a[i]);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    keep(s, sink);
}

__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 1/sqrt(x) converges to 1 from any positive start
__global__ void __launch_bounds__(kThreads) k_peak_rsqrt(float seed, int iters, float* sink)
{
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = seed * (i + 1) + 1e-6f * threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = rsqrt_ftz(a[i]);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    keep(s, sink);
}

// Random 16-byte loads; indices from a 32-bit LCG per thread, masked into the
// buffer, so every load is in bounds.
__global__ void __launch_bounds__(kThreads) k_peak_gather(const float4* __restrict__ buf, uint32_t mask, int iters,
                                                          float* sink)
{
    uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float4 v[kGatherLoads];
#pragma unroll
        for (int k = 0; k < kGatherLoads; ++k) {
            h = h * 1664525u + 1013904223u;
            v[k] = __ldg(buf + ((h >> 7) & mask));
        }
#pragma unroll
        for (int k = 0; k < kGatherLoads; ++k) acc += v[k].x + v[k].y + v[k].z + v[k].w;
    }
    keep(acc, sink);
}

int fail(adg_ctx* ctx, cudaError_t e, const char* what)
{
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return ADG_ECUDA;
}

}  // namespace

extern "C" int adg_probe_peaks(adg_ctx* ctx, adg_peaks* out)
{
    if (!ctx || !out) return ADG_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(ctx, e, "cudaSetDevice");
    int sms = 0, khz = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess)
        return fail(ctx, e, "cudaDeviceGetAttribute");
    if ((e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device)) != cudaSuccess)
        return fail(ctx, e, "cudaDeviceGetAttribute");
    float4* buf = nullptr;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double ms[5] = {0, 0, 0, 0, 0};
    const unsigned blocks = (unsigned)sms * kBlocksPerSm;
    const double threads = (double)blocks * kThreads;
    auto run = [&]() -> cudaError_t {
        cudaError_t r;
        if ((r = cudaMalloc(&buf, sizeof(float4) * kGatherElems)) != cudaSuccess) return r;
        if ((r = cudaMalloc(&sink, sizeof(float) * kThreads)) != cudaSuccess) return r;
        if ((r = cudaMemsetAsync(buf, 0, sizeof(float4) * kGatherElems, ctx->stream)) != cudaSuccess) return r;
        if ((r = cudaEventCreate(&e0)) != cudaSuccess) return r;
        if ((r = cudaEventCreate(&e1)) != cudaSuccess) return r;
        for (int p = 0; p < 5; ++p) {
            for (int rep = 0; rep < 2; ++rep) {  // the first launch is untimed
                if (rep == 1 && (r = cudaEventRecord(e0, ctx->stream)) != cudaSuccess) return r;
                if (p == 0) k_peak_fma<<<blocks, kThreads, 0, ctx->stream>>>(0.5f, kFmaIters, sink);
                else if (p == 1) k_peak_fma2<<<blocks, kThreads, 0, ctx->stream>>>(0.5f, kFmaIters / 2, sink);
                else if (p == 2) k_peak_ex2<<<blocks, kThreads, 0, ctx->stream>>>(0.5f, kEx2Iters, sink);
                else if (p == 3) k_peak_rsqrt<<<blocks, kThreads, 0, ctx->stream>>>(0.5f, kEx2Iters, sink);
                else k_peak_gather<<<blocks, kThreads, 0, ctx->stream>>>(buf, kGatherElems - 1, kGatherIters, sink);
                if ((r = cudaGetLastError()) != cudaSuccess) return r;
                if (rep == 1 && (r = cudaEventRecord(e1, ctx->stream)) != cudaSuccess) return r;
            }
            if ((r = cudaEventSynchronize(e1)) != cudaSuccess) return r;
            float t = 0.f;
            if ((r = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) return r;
            ms[p] = t;
        }
        return cudaSuccess;
    };
    e = run();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return fail(ctx, e, "peak probes");
    ctx->stats.kernel_launches += 10;
    const double fma_flops = threads * kFmaIters * (2.0 * kChains) * 2.0;  // FMA = 2 flops
    const double fma2_flops = threads * (kFmaIters / 2) * kChains * 2.0 * 2.0;
    out->fp32_scalar_tflops = fma_flops / (ms[0] * 1e-3) / 1e12;
    out->fp32x2_tflops = fma2_flops / (ms[1] * 1e-3) / 1e12;
    out->fp32_tflops = out->fp32_scalar_tflops > out->fp32x2_tflops ? out->fp32_scalar_tflops : out->fp32x2_tflops;
    out->mufu_gops = threads * kEx2Iters * kChains / (ms[2] * 1e-3) / 1e9;
    out->mufu_rsqrt_gops = threads * kEx2Iters * kChains / (ms[3] * 1e-3) / 1e9;
    out->l2_gather_gbs = threads * kGatherIters * kGatherLoads * 16.0 / (ms[4] * 1e-3) / 1e9;
    out->gather_bytes = (int64_t)sizeof(float4) * kGatherElems;
    out->sms = sms;
    out->sm_clock_mhz = khz / 1000;
    return ADG_OK;
}
