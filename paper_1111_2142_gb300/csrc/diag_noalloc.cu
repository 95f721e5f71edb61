// Allocation-free variant of the FP64 diagnostics reduction.
//
// lwacm_diagnostics() keeps its per-block partial sums in the workspace that the
// caller binds to a context. Some callers cannot hand out device memory at all:
// code that runs where cudaMalloc is forbidden or unavailable (inside a region
// that must not allocate, under an allocator that is locked, or from a tool that
// only owns the field arrays of a running simulation). For them this file keeps
// the partial sums in a fixed, file-scope device array instead, and the entry
// point allocates nothing: no cudaMalloc / cudaFree and no allocating library
// call. The caller passes the input fields and the device array that receives
// the result.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lwacm.h"
#include "lwacm_core.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 128;
constexpr long long kPerBlock = (long long)kThreads * kPerThread;  // 32768 nodes per block
constexpr int kMaxBlocks = 1024;                                   // LWACM_NOALLOC_MAX_N / kPerBlock
constexpr int kVals = 9;  // sum d, sum rho u (3), KE, max |u|^2, M_par, M_perp, non-finite count
constexpr int kMaxDevices = 64;

static_assert((long long)kMaxBlocks * kPerBlock == LWACM_NOALLOC_MAX_N, "capacity mismatch");

// Scratch for the per-block partial sums: 1024 x 9 doubles = 72 KiB. It lives in
// every GPU that loads this library until the process exits. All calls share it;
// each call overwrites the slots of the blocks it launches before the final
// pass reads them, so nothing has to start at zero.
static __device__ __align__(256) double g_partials[kMaxBlocks * kVals];

template <typename T>
__global__ void __launch_bounds__(kThreads) k_partials(const T *__restrict__ d, const T *__restrict__ ux,
                                                       const T *__restrict__ uy, const T *__restrict__ uz,
                                                       long long n, double *__restrict__ partial) {
    double acc[kVals] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const long long base = (long long)blockIdx.x * kPerBlock;
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + (long long)k * kThreads + threadIdx.x;
        if (i >= n) break;
        const double dd = lwacm::ldf(d + i), u = lwacm::ldf(ux + i), v = lwacm::ldf(uy + i);
        const double w = uz ? (double)lwacm::ldf(uz + i) : 0.0;
        const double rho = 1.0 + dd, uu = u * u + v * v + w * w;
        acc[0] += dd;
        acc[1] += rho * u;
        acc[2] += rho * v;
        acc[3] += rho * w;
        acc[4] += 0.5 * rho * uu;
        acc[5] = fmax(acc[5], uu);
        if (uz) {
            // Eq. 3Dmomenta, read for a lid moving along the x = y diagonal of the
            // top z plane: components parallel / perpendicular to the lid (times sqrt 2)
            acc[6] += 0.5 * (u + v) * (u + v);
            acc[7] += 0.5 * (u - v) * (u - v);
        }
        if (!isfinite(dd) || !isfinite(uu)) acc[8] += 1.0;
    }
    __shared__ double sh[kVals][kThreads];
    for (int q = 0; q < kVals; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int q = 0; q < kVals; ++q) {
                const double o = sh[q][threadIdx.x + off];
                sh[q][threadIdx.x] = q == 5 ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        __syncthreads();
    }
    if (threadIdx.x < kVals) partial[(long long)blockIdx.x * kVals + threadIdx.x] = sh[threadIdx.x][0];
}

// one block: the partials in a fixed order (deterministic), max |u|^2 -> max |u|
__global__ void __launch_bounds__(kThreads) k_final(const double *__restrict__ partial, int nblocks,
                                                    double *__restrict__ out) {
    __shared__ double sh[kVals][kThreads];
    double acc[kVals] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int q = 0; q < kVals; ++q) {
            const double o = partial[(long long)b * kVals + q];
            acc[q] = q == 5 ? fmax(acc[q], o) : acc[q] + o;
        }
    for (int q = 0; q < kVals; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int q = 0; q < kVals; ++q) {
                const double o = sh[q][threadIdx.x + off];
                sh[q][threadIdx.x] = q == 5 ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        __syncthreads();
    }
    if (threadIdx.x < kVals) out[threadIdx.x] = threadIdx.x == 5 ? sqrt(sh[5][0]) : sh[threadIdx.x][0];
}

// Host-side device address of g_partials, looked up once per device with that
// device current (the symbol's host-side name is not a device address), and kept
// until the process exits: a cudaDeviceReset() of the device would make it stale,
// which the header states as a limit of this entry point.
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

template <typename T>
cudaError_t run(const void *d, const void *ux, const void *uy, const void *uz, long long n, double *scratch,
                double *out, cudaStream_t st) {
    const int nb = (int)((n + kPerBlock - 1) / kPerBlock);
    k_partials<T><<<nb, kThreads, 0, st>>>((const T *)d, (const T *)ux, (const T *)uy, (const T *)uz, n,
                                           scratch);
    k_final<<<1, kThreads, 0, st>>>(scratch, nb, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" lwacm_status lwacm_diagnostics_noalloc(const void *d, const void *ux, const void *uy,
                                                  const void *uz, long long n, int dtype,
                                                  double *out_dev, void *stream) {
    if (!d || !ux || !uy || !out_dev) return LWACM_E_ARG;
    if (dtype != LWACM_F32 && dtype != LWACM_BF16 && dtype != LWACM_F16) return LWACM_E_ARG;
    if (n < 1) return LWACM_E_ARG;
    if (n > LWACM_NOALLOC_MAX_N) return LWACM_E_RANGE;  // more nodes than the scratch covers
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return LWACM_E_CUDA;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (dtype == LWACM_F32)
        e = run<float>(d, ux, uy, uz, n, scratch, out_dev, st);
    else if (dtype == LWACM_BF16)
        e = run<__nv_bfloat16>(d, ux, uy, uz, n, scratch, out_dev, st);
    else
        e = run<__half>(d, ux, uy, uz, n, scratch, out_dev, st);
    return e == cudaSuccess ? LWACM_OK : LWACM_E_CUDA;
}
