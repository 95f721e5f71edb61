// Register-only FP32 FMA throughput probe: the compute roof the LW-ACM kernels
// are placed against (their update is ~150 FP32 operations per node).
#include <cuda_runtime.h>

#include "../../include/lwacm.h"
#include "../../include/lwacm_measure.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;

__device__ float g_sink[1];

__global__ void __launch_bounds__(kThreads) k_ffma_chains(long long iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // b < 1 keeps every chain bounded near c/(1-b); the sum is never -1
    if (s == -1.f) g_sink[0] = s;
}

}  // namespace

extern "C" int lwacm_measure_fp32_peak(long long iters, void *stream, double *tflops, double *ms) {
    if (!tflops || !ms || iters < 1 || iters > (1LL << 20)) return LWACM_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LWACM_E_CUDA;
    const unsigned grid = (unsigned)(sms * kCtasPerSm);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LWACM_OK;
    float t = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = LWACM_E_CUDA;
    } else {
        k_ffma_chains<<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f);
        cudaEventRecord(e0, st);
        k_ffma_chains<<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            rc = LWACM_E_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != LWACM_OK) return rc;
    const double fma = (double)grid * kThreads * kChains * kUnroll * (double)iters;
    *ms = t;
    *tflops = 2.0 * fma / (t * 1e-3) / 1e12;
    return LWACM_OK;
}
