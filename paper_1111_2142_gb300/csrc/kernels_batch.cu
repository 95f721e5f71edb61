// Batched update of many independent periodic domains of different sizes and
// viscosities, packed one after the other in the same field arrays.
//
// The domains are cut into tiles of 256 consecutive nodes (a tile never spans two
// domains); a CTA walks the tile list with a grid stride, one node per thread,
// and updates it with the per-node moment form of Eq. ACM2.0 (node_update.cuh)
// using its domain's (nx, ny, nz, nu).
//
//   k_batch_step        one launch = one step of every domain (the host replays
//                       the steps from captured CUDA graphs);
//   k_batch_persistent  one cooperative launch runs all the steps: the CTAs meet
//                       at a grid-wide barrier between steps. The barrier spins a
//                       bounded number of times; a CTA that gives up sets the
//                       device error word to 2 and returns, so a missing arrival
//                       ends the launch instead of hanging it.
#include <cooperative_groups.h>

#include "launch.h"
#include "lwacm_core.cuh"
#include "node_update.cuh"

namespace lwacm {
namespace {

constexpr int kTile = 256;
constexpr int kBarrierPolls = 1 << 21;  // with 256 ns back-off: well under a second

template <int Q, typename T>
__device__ __forceinline__ void tile_update(const T *__restrict__ in, T *__restrict__ out,
                                            const BatchParams &bp, long long t) {
    const BatchTile tile = bp.tiles[t];
    const BatchDomain dm = bp.doms[tile.dom];
    const long long k = tile.start + threadIdx.x;
    if (k >= dm.off + dm.n) return;
    const long long local = k - dm.off;
    StepParams p;
    p.nx = dm.nx;
    p.ny = dm.ny;
    p.nz = dm.nz;
    p.bc = BC_PERIODIC;
    p.N = dm.n;
    p.fstride = bp.fstride;
    p.s = dm.s;
    p.a = dm.a;
    p.wallc = 0.f;
    p.has_force = 0;
    p.gfield = nullptr;
    p.lid_axis = 0;
    p.err = nullptr;
    for (int c = 0; c < 3; ++c) {
        p.lid[c] = 0.f;
        p.force[c] = 0.f;
        p.walled[c] = 0;
    }
    const int x = (int)(local % dm.nx);
    const long long r = local / dm.nx;
    const int y = (int)(r % dm.ny);
    const int z = (int)(r / dm.ny);
    node_update<Q, false>(in + dm.off, out + dm.off, p, x, y, z);
}

template <int Q, typename T>
__global__ void __launch_bounds__(kTile) k_batch_step(const T *__restrict__ in, T *__restrict__ out,
                                                      BatchParams bp) {
    for (long long t = blockIdx.x; t < bp.ntiles; t += gridDim.x) tile_update<Q, T>(in, out, bp, t);
}

// Grid-wide barrier number `gen` (1, 2, ...): arrive on a counter, the last CTA
// resets it and publishes the generation; the others poll it, bounded.
__device__ bool grid_barrier(const BatchParams &bp, unsigned gen) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned arrived = atomicAdd(bp.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bp.bar_count, 0u);
            __threadfence();
            atomicExch(bp.bar_gen, gen);
        } else {
            ok = 0;
            for (int it = 0; it < kBarrierPolls; ++it) {
                if (atomicAdd(bp.bar_gen, 0u) >= gen) {
                    ok = 1;
                    break;
                }
                __nanosleep(256);
            }
            if (!ok) atomicExch(bp.err, 2);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <int Q, typename T>
__global__ void __launch_bounds__(kTile) k_batch_persistent(T *buf0, T *buf1, BatchParams bp,
                                                            long long nsteps, int parity) {
    for (long long s = 0; s < nsteps; ++s) {
        const int cur = (int)((parity + s) & 1);
        const T *in = cur ? buf1 : buf0;
        T *out = cur ? buf0 : buf1;
        for (long long t = blockIdx.x; t < bp.ntiles; t += gridDim.x) tile_update<Q, T>(in, out, bp, t);
        if (s + 1 < nsteps) {
            // test hook: CTA 0 leaves without arriving, so the others' waits run out
            if (bp.withhold_step == s && blockIdx.x == 0) return;
            if (!grid_barrier(bp, (unsigned)(s + 1))) return;
        }
    }
}

template <int Q, typename T>
cudaError_t persistent_t(void *b0, void *b1, const BatchParams &bp, long long nsteps, int parity,
                         cudaStream_t st) {
    static int max_ctas = 0;
    if (max_ctas == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_persistent<Q, T>, kTile, 0);
        if (e != cudaSuccess) return e;
        max_ctas = per * sms;
        if (max_ctas < 1) return cudaErrorNotSupported;
    }
    const long long grid = bp.ntiles < max_ctas ? bp.ntiles : max_ctas;
    T *p0 = (T *)b0, *p1 = (T *)b1;
    BatchParams q = bp;
    void *args[] = {&p0, &p1, &q, &nsteps, &parity};
    return cudaLaunchCooperativeKernel((const void *)k_batch_persistent<Q, T>, dim3((unsigned)grid), dim3(kTile),
                                       args, 0, st);
}

template <typename T>
cudaError_t step_t(int Q, const void *in, void *out, const BatchParams &bp, cudaStream_t st) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 152;
    }
    const long long cap = (long long)sms * 8;
    const unsigned grid = (unsigned)(bp.ntiles < cap ? bp.ntiles : cap);
    if (Q == 9)
        k_batch_step<9, T><<<grid, kTile, 0, st>>>((const T *)in, (T *)out, bp);
    else
        k_batch_step<19, T><<<grid, kTile, 0, st>>>((const T *)in, (T *)out, bp);
    return cudaGetLastError();
}

}  // namespace

int batch_tile() { return kTile; }

cudaError_t launch_batch_step(int Q, int storage, const void *in, void *out, const BatchParams &bp,
                              cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return step_t<float>(Q, in, out, bp, st);
        case STORE_BF16: return step_t<__nv_bfloat16>(Q, in, out, bp, st);
        case STORE_F16: return step_t<__half>(Q, in, out, bp, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_persistent(int Q, int storage, void *buf0, void *buf1, const BatchParams &bp,
                                    long long nsteps, int parity, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bp.bar_count, 0, 2 * sizeof(unsigned), st);  // count, generation
    if (e != cudaSuccess) return e;
    if (Q == 9) {
        switch (storage) {
            case STORE_F32: return persistent_t<9, float>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_BF16: return persistent_t<9, __nv_bfloat16>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_F16: return persistent_t<9, __half>(buf0, buf1, bp, nsteps, parity, st);
        }
    } else {
        switch (storage) {
            case STORE_F32: return persistent_t<19, float>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_BF16: return persistent_t<19, __nv_bfloat16>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_F16: return persistent_t<19, __half>(buf0, buf1, bp, nsteps, parity, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lwacm
