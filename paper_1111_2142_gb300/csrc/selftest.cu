// Device self-tests of the kernels' numerical building blocks.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lwacm.h"
#include "../../include/lwacm_selftest.h"
#include "tile_common.cuh"

namespace {

__global__ void k_reciprocal(const float *__restrict__ x, float *__restrict__ out, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = lwacm::tile::rcp_nr(x[k]);
}

}  // namespace

extern "C" int lwacm_selftest_reciprocal(const float *x_dev, float *out_dev, long long n, void *stream) {
    if (!x_dev || !out_dev || n < 1 || n >= (1LL << 31)) return LWACM_E_ARG;
    const long long blocks = (n + 255) / 256;
    const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
    k_reciprocal<<<grid, 256, 0, (cudaStream_t)stream>>>(x_dev, out_dev, n);
    return cudaGetLastError() == cudaSuccess ? LWACM_OK : LWACM_E_CUDA;
}
