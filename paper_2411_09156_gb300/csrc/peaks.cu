// Throughput microbenchmarks that give the roofline denominators of the render
// kernels, which are bound by instruction issue rather than by HBM: FP32 fused
// multiply-add, the special-function unit (ex2 and rcp, the approximations the
// render uses) and FP32 atomic adds into L2 in the render backward's pattern (16
// lanes of a warp on one 64-byte line). They are a measurement utility of the
// library, not part of the method. Each kernel runs many independent chains per
// thread so that latency is hidden and the pipe's throughput shows.
#include "ges_internal.cuh"

namespace ges {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;   // independent dependency chains per thread
constexpr int kUnroll = 16;  // chain steps per loop iteration

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(int iters, float *sink) {
    float c[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = 1e-3f * (float)(threadIdx.x + k);
    const float m = 0.9999999f, d = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) c[k] = __fmaf_rn(c[k], m, d);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += c[k];
    if (s == -1.f) sink[threadIdx.x] = s;  // never true; keeps the chains live
}

// ex2 chain x <- 2^-x stays in [1/2, 1]; rcp chain x <- 1 / (x + 1) converges to 0.618 (the add
// keeps the compiler from pairing reciprocals away and runs on the FMA pipe, 4x wider).
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak_mufu(int iters, float *sink) {
    float c[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = 0.5f + 1e-3f * (float)((threadIdx.x + k) & 63);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) c[k] = KIND == 1 ? ex2_approx(-c[k]) : rcp_approx(c[k] + 1.f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += c[k];
    if (s == -1.f) sink[threadIdx.x] = s;
}

// Each warp adds into `iters` lines spread over the buffer by a multiplicative hash, 16 lanes
// on one 64-byte line per instruction (the backward's coalesced accumulator update).
__global__ void __launch_bounds__(kPeakThreads) k_peak_atomic(int iters, float *lines, uint32_t n_lines) {
    const uint32_t warp = (blockIdx.x * kPeakThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < iters; ++i) {
        const uint32_t line = (warp * 2654435761u + (uint32_t)i * 40503u) % n_lines;
        if (lane < 16) atomicAdd(lines + 16 * (size_t)line + lane, 1.0f);
    }
}

}  // namespace
}  // namespace ges

using namespace ges;

ges_status ges_peak_run(int32_t kind, int32_t blocks_per_sm, int32_t iters, float *sink, uint64_t sink_floats,
                        void *stream, uint64_t *ops) {
    GES_RANGE();
    if (kind < 0 || kind > 3 || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !sink || !ops)
        return GES_ERR_INVALID_ARG;
    if (sink_floats < (uint64_t)kPeakThreads) return GES_ERR_INVALID_ARG;
    if (kind == 3 && (sink_floats % 16 != 0 || sink_floats / 16 > 0xffffffffull)) return GES_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GES_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GES_ERR_CUDA;
    const int grid = sms * blocks_per_sm;
    const uint64_t threads = (uint64_t)grid * kPeakThreads;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case 0:
            k_peak_fma<<<grid, kPeakThreads, 0, s>>>(iters, sink);
            *ops = threads * (uint64_t)iters * kUnroll * kChains * 2;  // flops: an FMA is two
            break;
        case 1:
            k_peak_mufu<1><<<grid, kPeakThreads, 0, s>>>(iters, sink);
            *ops = threads * (uint64_t)iters * kUnroll * kChains;
            break;
        case 2:
            k_peak_mufu<2><<<grid, kPeakThreads, 0, s>>>(iters, sink);
            *ops = threads * (uint64_t)iters * kUnroll * kChains;
            break;
        default:
            k_peak_atomic<<<grid, kPeakThreads, 0, s>>>(iters, sink, (uint32_t)(sink_floats / 16));
            *ops = threads / 32 * (uint64_t)iters * 16;
            break;
    }
    return cudaGetLastError() == cudaSuccess ? GES_OK : GES_ERR_CUDA;
}
