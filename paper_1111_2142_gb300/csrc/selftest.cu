// Self-tests of the kernels' numerical building blocks (device) and of the
// row-tiled kernels' work schedule (host).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lwacm.h"
#include "../../include/lwacm_selftest.h"
#include "tile_common.cuh"

namespace {

// packed 1: element pairs (2k, 2k+1) through the FP32x2 form the half-row kernel
// uses (an odd last element through the scalar form); 2: the reciprocal of b that
// form divides with; 0: every element through the scalar form
__global__ void k_quotient(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ out,
                           long long n, int packed) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (packed == 2) {  // the reciprocal RN(1/b) itself (a unused), FP32x2 form
        for (long long k = t0; k < n / 2; k += stride) {
            const float2 y = lwacm::tile::div_prep2(make_float2(b[2 * k], b[2 * k + 1])).y;
            out[2 * k] = y.x;
            out[2 * k + 1] = y.y;
        }
        if ((n & 1) && t0 == 0) out[n - 1] = lwacm::tile::rcp_rn(b[n - 1]);
    } else if (packed) {
        const long long np = n / 2;
        for (long long k = t0; k < np; k += stride) {
            const float2 a2 = make_float2(a[2 * k], a[2 * k + 1]);
            const float2 b2 = make_float2(b[2 * k], b[2 * k + 1]);
            const float2 q = lwacm::tile::div_apply2(a2, lwacm::tile::div_prep2(b2));
            out[2 * k] = q.x;
            out[2 * k + 1] = q.y;
        }
        if ((n & 1) && t0 == 0) out[n - 1] = lwacm::tile::div_apply(a[n - 1], lwacm::tile::div_prep(b[n - 1]));
    } else {
        for (long long k = t0; k < n; k += stride)
            out[k] = lwacm::tile::div_apply(a[k], lwacm::tile::div_prep(b[k]));
    }
}

// stochastic rounding of x[k] as the half-row kernel stores field 0 (the density) of
// node k in the step with counter `step`, widened back to FP32; four elements per
// call of the kernel's store routine
template <typename T>
__global__ void k_round(const float *__restrict__ x, float *__restrict__ out, long long n, uint32_t key) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x); k < n; k += 4 * stride) {
        float v[4];
        uint32_t h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[i] = k + i < n ? x[k + i] : 0.f;
            h[i] = lwacm::tile::sr_bits((uint32_t)(k + i), 0u, key);
        }
        __align__(8) T t[4];
        lwacm::tile::st4_sr(t, v[0], v[1], v[2], v[3], h[0], h[1], h[2], h[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (k + i < n) out[k + i] = (float)t[i];
    }
}

}  // namespace

extern "C" int lwacm_selftest_round(const float *x_dev, float *out_dev, long long n, int storage, unsigned step,
                                    void *stream) {
    if (!x_dev || !out_dev || n < 1 || n >= (1LL << 31) || (storage != LWACM_BF16 && storage != LWACM_F16))
        return LWACM_E_ARG;
    const long long blocks = (n + 1023) / 1024;
    const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
    const uint32_t key = lwacm::tile::sr_key(step);
    if (storage == LWACM_BF16)
        k_round<__nv_bfloat16><<<grid, 256, 0, (cudaStream_t)stream>>>(x_dev, out_dev, n, key);
    else
        k_round<__half><<<grid, 256, 0, (cudaStream_t)stream>>>(x_dev, out_dev, n, key);
    return cudaGetLastError() == cudaSuccess ? LWACM_OK : LWACM_E_CUDA;
}

extern "C" int lwacm_selftest_quotient(const float *a_dev, const float *b_dev, float *out_dev, long long n,
                                       int packed, void *stream) {
    if (!a_dev || !b_dev || !out_dev || n < 1 || n >= (1LL << 31) || packed < 0 || packed > 2) return LWACM_E_ARG;
    const long long blocks = (n + 255) / 256;
    const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
    k_quotient<<<grid, 256, 0, (cudaStream_t)stream>>>(a_dev, b_dev, out_dev, n, packed == 2 ? 2 : (packed ? 1 : 0));
    return cudaGetLastError() == cudaSuccess ? LWACM_OK : LWACM_E_CUDA;
}

extern "C" int lwacm_selftest_schedule(int cols, int nz, int ctas, int *grid, int *zc, int *kcls, int *items,
                                       long long cap, long long *count) {
    if (cols < 1 || nz < 1 || ctas < 1 || (long long)cols * nz >= (1LL << 31) || !grid || !zc || !kcls || !count ||
        cap < 0 || (cap > 0 && !items))
        return LWACM_E_ARG;
    const lwacm::tile::Schedule sc = lwacm::tile::plan_schedule(cols, nz, ctas);
    *grid = sc.grid;
    *zc = sc.zc;
    *kcls = sc.kcls;
    long long n = 0;
    for (int b = 0; b < sc.grid && b < sc.nitems; ++b) {  // CTAs b >= nitems return at once
        lwacm::tile::TaskIter it(b, sc.nitems, sc.grid, cols, sc.zc, nz, sc.kcls);
        while (it.valid()) {
            if (n < cap) {
                items[4 * n] = b;
                items[4 * n + 1] = it.col;
                items[4 * n + 2] = it.za;
                items[4 * n + 3] = it.zb;
            }
            ++n;
            do {  // through the item's source planes, as the kernel steps, to the next item
                it.next();
            } while (it.valid() && it.pz != it.za - 1);
        }
    }
    *count = n;
    return LWACM_OK;
}
