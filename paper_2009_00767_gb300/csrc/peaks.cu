// peaks.cu -- throughput probes for the roofline denominators of the arithmetic-bound stages: the
// FP32 FMA pipe (P2M and L2P power chains), the MUFU lg2 unit (the near field's logarithms) and the
// FP64 FMA pipe (the plain path).  Each thread runs independent dependency chains (8 for the FMA
// pipes; 32 for lg2, whose latency is several times longer), over a grid of eight 256-thread
// blocks per SM, so that latency does not set the rate; the rate is the best of three timed launches
// on the caller's stream.
#include <cuda_runtime.h>

#include "fmm_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kLg2Chains = 32;
constexpr int kBlocksPerSm = 8;
constexpr int kThreadsPerBlock = 256;

// x <- x a + b: with a = 1 - 2^-10 and b = 2^-10 every chain stays near 1, so nothing overflows
__global__ void k_probe_ffma(int iters, float a, float b, float* sink) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.0f) sink[0] = s;   // never true: keeps the chains from being removed
}

// x <- lg2(x) + c: with c = 2 every chain stays near the fixed point 4 (lg2 4 = 2); the add runs on
// the FMA pipe, four times faster than the MUFU unit, so the MUFU unit sets the rate
__global__ void k_probe_lg2(int iters, float c, float* sink) {
    float x[kLg2Chains];
#pragma unroll
    for (int i = 0; i < kLg2Chains; ++i) x[i] = 3.0f + 0.01f * (float)i + 1e-4f * (float)threadIdx.x;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kLg2Chains; ++i) {
            float r;
            asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[i]));
            x[i] = r + c;
        }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kLg2Chains; ++i) s += x[i];
    if (s == -1.0f) sink[0] = s;
}

__global__ void k_probe_dfma(int iters, double a, double b, float* sink) {
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0 + 1e-3 * (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.0) sink[0] = (float)s;
}

}  // namespace

extern "C" fmm_status fmm_probe_peak(int unit, double* ops_per_s, void* stream) {
    if (ops_per_s == nullptr || unit < FMM_PROBE_FP32_FMA || unit > FMM_PROBE_FP64_FMA) return FMM_ERR_INVALID_ARG;
    *ops_per_s = 0.0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FMM_ERR_CUDA;
    const unsigned blocks = (unsigned)(sms * kBlocksPerSm);
    const double threads = (double)blocks * kThreadsPerBlock;
    // iterations sized for a few milliseconds per launch on a GB300
    const int iters = unit == FMM_PROBE_FP32_FMA ? 32768 : (unit == FMM_PROBE_MUFU_LG2 ? 2048 : 2048);
    const double per_thread =
        unit == FMM_PROBE_MUFU_LG2 ? (double)iters * kLg2Chains : (double)iters * kChains * 2.0;   // FMA = 2 flop
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fmm_status rc = FMM_OK;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return FMM_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FMM_ERR_CUDA;
    double best = 0.0;
    for (int rep = 0; rep < 4 && rc == FMM_OK; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, st);
        if (unit == FMM_PROBE_FP32_FMA)
            k_probe_ffma<<<blocks, kThreadsPerBlock, 0, st>>>(iters, 1.0f - 0x1p-10f, 0x1p-10f, sink);
        else if (unit == FMM_PROBE_MUFU_LG2)
            k_probe_lg2<<<blocks, kThreadsPerBlock, 0, st>>>(iters, 2.0f, sink);
        else
            k_probe_dfma<<<blocks, kThreadsPerBlock, 0, st>>>(iters, 1.0 - 0x1p-10, 0x1p-10, sink);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = FMM_ERR_CUDA;
            break;
        }
        if (rep > 0 && ms > 0.f) best = fmax(best, threads * per_thread / (ms * 1e-3));
    }
    if (rc == FMM_OK && cudaGetLastError() != cudaSuccess) rc = FMM_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc == FMM_OK) *ops_per_s = best;
    return rc;
}
