// Tiled interior kernel for D3Q19 on periodic domains with nx = 32*VX (VX = 4, 8)
// and ny a multiple of 8: the moment form of Eq. ACM2.0 (see lwacm_core.cuh), every
// field read from HBM once and written once per step.
//
// Persistent CTAs (one per SM) of 8 warps. The (y-column, z) plane-rows of the
// lattice (a y-column is 8 consecutive rows) are split into equal contiguous
// ranges, one per CTA; a CTA marches along z through its range, one source plane
// per task. Per plane:
//   * TMA (cp.async.bulk, mbarrier completion, two-stage ring) copies the ten rows
//     y0-1 .. y0+8 of the four fields into shared memory two tasks ahead;
//   * warp w owns row y0+w, lane l the VX consecutive nodes x = l*VX + i; each node
//     computes its outgoing values g_i once (pre-combine, Eq. ACM2.0b(a)) and
//     streams them (Eq. ACM2.0b(b)): links with c_y = 0 stay in the warp (register
//     moves, one shuffle at lane edges, periodic in x through lane 31 -> 0); links
//     with c_y = +-1 are summed per receiver into four values and passed through
//     shared memory to the next / previous row (double-buffered, one CTA barrier
//     per plane); warps 0 and 7 also compute those values for the halo rows
//     y0-1 and y0+8;
//   * links with c_z = +-1 land in register accumulators of planes z+-1 (three
//     planes of (d, jx, jy, jz) rotate); plane z-1 is then complete, post-combined
//     (+ a rho u, Eq. ACM2.0b(c)), divided by rho (moments, Section 2.1) and
//     stored with 16-byte stores.
// The first and last plane of a run (the z-halo) only evaluate the five links that
// point into the run.
// Every wait on an mbarrier is bounded; on timeout the CTA sets an error word,
// waits (bounded) for its own copies in flight and exits.
#include <stdint.h>

#include "dev_cache.h"
#include "launch.h"
#include "lwacm_core.cuh"
#include "tile_common.cuh"

namespace lwacm {
namespace {

using namespace tile;


constexpr int NTHREADS = ROWS * 32;

template <int VX>
struct Geo {
    static constexpr int RL = 32 * VX;                   // row length (floats)
    static constexpr int XSLOT = ROWS * RL;              // one slot, all receiver rows
    static constexpr int XDIR = NSLOT * XSLOT;
    static constexpr int XBUF = 2 * XDIR;                // up + down
    static constexpr int STAGE = 4 * TROWS * RL;         // 4 fields x 10 rows
    static constexpr size_t XBYTES = 2 * (size_t)XBUF * 4;   // double-buffered exchange
    static constexpr size_t SBYTES = 2 * (size_t)STAGE * 4;  // two TMA stages
    static constexpr size_t BYTES = XBYTES + SBYTES + 64;    // + mbarriers
    static constexpr uint32_t TX = STAGE * 4;                // bytes per stage
};

// Row-crossing values of one row for the receivers above (UP, c_y = +1) or below
// (c_y = -1), four per receiver x:
//   slot 0: sum of the three c_z = 0 links  (d, and +-jy)
//   slot 1: their x-momentum                (jx)
//   slot 2: the c_z = +1 link               (plane ahead)
//   slot 3: the c_z = -1 link               (plane behind)
// MODE FIRST needs slot 2 only, LAST slot 3 only.
template <int VX, int MODE, bool UP>
__device__ __forceinline__ void send_row(const NodeConst<VX> &nc, float c4, float *xdir, int row,
                                         int lane) {
    using G = Geo<VX>;
    float *base = xdir + row * G::RL;
    if (MODE == MID) {
        float s0[VX], s1[VX];
        {  // k = 0: c = (0,1,0), -c = (0,-1,0)
            float gp[VX], gm[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) pair_g(nc, i, ypair_e(nc, 0, i), false, gp[i], gm[i]);
#pragma unroll
            for (int i = 0; i < VX; ++i) s0[i] = UP ? gp[i] : gm[i];
        }
        {  // k = 1: c = (1,1,0) [up: receiver x <- x-1]; -c = (-1,-1,0) [down: x <- x+1]
            float gp[VX], gm[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) pair_g(nc, i, ypair_e(nc, 1, i), true, gp[i], gm[i]);
            if (UP) {
                xshift(gp, 1, lane);
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    s0[i] += gp[i];
                    s1[i] = gp[i];
                }
            } else {
                xshift(gm, -1, lane);
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    s0[i] += gm[i];
                    s1[i] = -gm[i];
                }
            }
        }
        {  // k = 2: c = (-1,1,0) [up: x <- x+1]; -c = (1,-1,0) [down: x <- x-1]
            float gp[VX], gm[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) pair_g(nc, i, ypair_e(nc, 2, i), true, gp[i], gm[i]);
            if (UP) {
                xshift(gp, -1, lane);
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    s0[i] += gp[i];
                    s1[i] -= gp[i];
                }
            } else {
                xshift(gm, 1, lane);
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    s0[i] += gm[i];
                    s1[i] += gm[i];
                }
            }
        }
        st_slot(base + 0 * G::XSLOT, s0, lane);
        st_slot(base + 1 * G::XSLOT, s1, lane);
    }
    // k = 3: c = (0,1,1), -c = (0,-1,-1); k = 4: c = (0,1,-1), -c = (0,-1,1)
    if (MODE != LAST) {  // slot 2 (c_z = +1): up -> c of k = 3; down -> -c of k = 4
        float gp[VX], gm[VX];
        const int k = UP ? 3 : 4;
#pragma unroll
        for (int i = 0; i < VX; ++i) pair_g(nc, i, ypair_e(nc, k, i), true, gp[i], gm[i]);
        st_slot(base + 2 * G::XSLOT, UP ? gp : gm, lane);
    }
    if (MODE != FIRST) {  // slot 3 (c_z = -1): up -> c of k = 4; down -> -c of k = 3
        float gp[VX], gm[VX];
        const int k = UP ? 4 : 3;
#pragma unroll
        for (int i = 0; i < VX; ++i) pair_g(nc, i, ypair_e(nc, k, i), true, gp[i], gm[i]);
        st_slot(base + 3 * G::XSLOT, UP ? gp : gm, lane);
    }
}

// Phase A of a task: values of the staged source plane -> own accumulators and
// the exchange buffer.
template <int VX, int MODE, int PM, int P0, int PP>
__device__ __forceinline__ void phase_a(float (&acc)[3][VX][4], const float *stg, float *xbuf,
                                        const TiledParams &p, int lane, int warp) {
    using G = Geo<VX>;
    float *up = xbuf, *dn = xbuf + G::XDIR;
    {
        NodeConst<VX> nc;
        node_consts(nc, stg + (warp + 1) * G::RL, TROWS * G::RL, lane, p.s18);
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            float gp, gm;
            pair_g(nc, i, nc.W[i], false, gp, gm);  // (0,0,+1) / (0,0,-1)
            if (MODE == MID) {
                acc[P0][i][3] = acc[P0][i][0];  // jz so far = d so far (c_z = +1 arrivals)
                acc[P0][i][0] += 6.f * nc.K1[i];  // rest link: w_0 K = K/3
                const float ar = p.a_s * nc.A1[i];  // a rho (post-combine)
                acc[P0][i][1] = fmaf(ar, nc.U[i], acc[P0][i][1]);
                acc[P0][i][2] = fmaf(ar, nc.V[i], acc[P0][i][2]);
                acc[P0][i][3] = fmaf(ar, nc.W[i], acc[P0][i][3]);
            }
            if (MODE != LAST) acc[PP][i][0] += gp;
            if (MODE != FIRST) dep(acc[PM][i], gm, 0, 0, -1);
        }
        // in-row pairs c = (1,0,cz) / -c = (-1,0,-cz)
#pragma unroll
        for (int cz = -1; cz <= 1; ++cz) {
            // c lands in plane cz, -c in plane -cz: FIRST keeps only the plane ahead,
            // LAST only the plane behind
            const bool need_p = MODE == MID || (MODE == FIRST ? cz > 0 : cz < 0);
            const bool need_m = MODE == MID || (MODE == FIRST ? cz < 0 : cz > 0);
            if (!need_p && !need_m) continue;
            float eP = 0.f, eM = 0.f;
#pragma unroll
            for (int i = 0; i < VX; ++i) {
                float gp, gm;
                const float e = cz == 0 ? nc.U[i] : (cz > 0 ? nc.U[i] + nc.W[i] : nc.U[i] - nc.W[i]);
                pair_g(nc, i, e, cz != 0, gp, gm);
                if (need_p) {
                    if (i + 1 < VX)
                        dep(acc[pl<PM, P0, PP>(cz)][i + 1], gp, 1, 0, cz);
                    else
                        eP = gp;
                }
                if (need_m) {
                    if (i > 0)
                        dep(acc[pl<PM, P0, PP>(-cz)][i - 1], gm, -1, 0, -cz);
                    else
                        eM = gm;
                }
            }
            if (need_p) {
                const float rP = __shfl_sync(FULL, eP, (lane + 31) & 31);
                dep(acc[pl<PM, P0, PP>(cz)][0], rP, 1, 0, cz);
            }
            if (need_m) {
                const float rM = __shfl_sync(FULL, eM, (lane + 1) & 31);
                dep(acc[pl<PM, P0, PP>(-cz)][VX - 1], rM, -1, 0, -cz);
            }
        }
        if (warp + 1 < ROWS) send_row<VX, MODE, true>(nc, p.c4, up, warp + 1, lane);
        if (warp > 0) send_row<VX, MODE, false>(nc, p.c4, dn, warp - 1, lane);
    }
    // halo rows: y0-1 (staged row 0) feeds row 0, y0+8 (staged row 9) feeds row 7
    if (warp == 0) {
        NodeConst<VX> hc;
        node_consts(hc, stg, TROWS * G::RL, lane, p.s18);
        send_row<VX, MODE, true>(hc, p.c4, up, 0, lane);
    } else if (warp == ROWS - 1) {
        NodeConst<VX> hc;
        node_consts(hc, stg + (TROWS - 1) * G::RL, TROWS * G::RL, lane, p.s18);
        send_row<VX, MODE, false>(hc, p.c4, dn, ROWS - 1, lane);
    }
}

// Phase B: receive the row-crossing values; plane zfin (>= 0) is then complete and
// is stored.
template <int VX, int MODE, int PM, int P0, int PP>
__device__ __forceinline__ void phase_b(float (&acc)[3][VX][4], const float *xbuf, float *out,
                                        const TiledParams &p, int lane, int warp, int col,
                                        int zfin) {
    using G = Geo<VX>;
    const float *up = xbuf + warp * G::RL, *dn = xbuf + G::XDIR + warp * G::RL;
    float o[VX];
    if (MODE == MID) {
        ld_slot(up, o, lane);  // from below, c_z = 0: d, +jy
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            acc[P0][i][0] += o[i];
            acc[P0][i][2] += o[i];
        }
        ld_slot(up + G::XSLOT, o, lane);
#pragma unroll
        for (int i = 0; i < VX; ++i) acc[P0][i][1] += o[i];
        ld_slot(dn, o, lane);  // from above, c_z = 0: d, -jy
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            acc[P0][i][0] += o[i];
            acc[P0][i][2] -= o[i];
        }
        ld_slot(dn + G::XSLOT, o, lane);
#pragma unroll
        for (int i = 0; i < VX; ++i) acc[P0][i][1] += o[i];
    }
    if (MODE != LAST) {  // c_z = +1 arrivals for the plane ahead (jz implied by d)
        ld_slot(up + 2 * G::XSLOT, o, lane);
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            acc[PP][i][0] += o[i];
            acc[PP][i][2] += o[i];
        }
        ld_slot(dn + 2 * G::XSLOT, o, lane);
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            acc[PP][i][0] += o[i];
            acc[PP][i][2] -= o[i];
        }
    }
    if (MODE != FIRST) {  // c_z = -1 arrivals complete the plane behind
        ld_slot(up + 3 * G::XSLOT, o, lane);
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            acc[PM][i][0] += o[i];
            acc[PM][i][2] += o[i];
            acc[PM][i][3] -= o[i];
        }
        ld_slot(dn + 3 * G::XSLOT, o, lane);
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            acc[PM][i][0] += o[i];
            acc[PM][i][2] -= o[i];
            acc[PM][i][3] -= o[i];
        }
        if (zfin >= 0) {
            const long long rowoff = ((long long)zfin * p.ny + col * ROWS + warp) * p.nx + lane * VX;
            float *op = out + rowoff;
            float r[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) r[i] = __frcp_rn(1.f + acc[PM][i][0]);
#pragma unroll
            for (int h = 0; h < VX / 4; ++h) {
#define LW_ST(F, C, SC)                                                                         \
    reinterpret_cast<float4 *>(op + (F) * p.fstride)[h] =                                       \
        make_float4(acc[PM][4 * h][C] * (SC ? r[4 * h] : 1.f),                                  \
                    acc[PM][4 * h + 1][C] * (SC ? r[4 * h + 1] : 1.f),                          \
                    acc[PM][4 * h + 2][C] * (SC ? r[4 * h + 2] : 1.f),                          \
                    acc[PM][4 * h + 3][C] * (SC ? r[4 * h + 3] : 1.f))
                LW_ST(0, 0, false);
                LW_ST(1, 1, true);
                LW_ST(2, 2, true);
                LW_ST(3, 3, true);
#undef LW_ST
            }
        }
#pragma unroll
        for (int i = 0; i < VX; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[PM][i][c] = 0.f;
    }
}

// issue the TMA copies of the ten staged rows of source plane z of column col
template <int VX>
__device__ __forceinline__ void issue_plane(const float *in, const TiledParams &p, int col, int z,
                                            float *stage, uint64_t *bar) {
    using G = Geo<VX>;
    const int zl = z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z);
    const int y0 = col * ROWS;
    const long long plane = (long long)p.nx * p.ny;
    mbar_expect_tx(bar, G::TX);
    const uint32_t rb = (uint32_t)(G::RL * 4);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const float *src = in + f * p.fstride + (long long)zl * plane;
        float *dst = stage + f * TROWS * G::RL;
        if (y0 >= 1 && y0 + ROWS < p.ny) {
            bulk_g2s(dst, src + (long long)(y0 - 1) * p.nx, TROWS * rb, bar);
        } else {
            const int yb = y0 - 1 < 0 ? y0 - 1 + p.ny : y0 - 1;
            const int yt = y0 + ROWS >= p.ny ? y0 + ROWS - p.ny : y0 + ROWS;
            bulk_g2s(dst, src + (long long)yb * p.nx, rb, bar);
            bulk_g2s(dst + G::RL, src + (long long)y0 * p.nx, ROWS * rb, bar);
            bulk_g2s(dst + (TROWS - 1) * G::RL, src + (long long)yt * p.nx, rb, bar);
        }
    }
}

// After a MID plane, plane z-1 has been stored and zeroed: shift the window so
// that index 0 is again the plane behind, 1 the current plane, 2 the plane ahead.
template <int VX>
__device__ __forceinline__ void rotate(float (&acc)[3][VX][4]) {
#pragma unroll
    for (int i = 0; i < VX; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[0][i][c] = acc[1][i][c];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[1][i][c] = acc[2][i][c];  // jz of the plane ahead is implied
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[2][i][c] = 0.f;
    }
}

template <int VX>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_d3q19_tiled(const float *__restrict__ in, float *__restrict__ out, TiledParams p) {
    using G = Geo<VX>;
    extern __shared__ float4 smem4[];
    float *xs = reinterpret_cast<float *>(smem4);
    float *stg = xs + 2 * G::XBUF;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg + 2 * G::STAGE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if ((int)blockIdx.x >= p.nitems) return;  // uniform per CTA

    __shared__ int failed;
    if (threadIdx.x == 0) {
        failed = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    TaskIter it(blockIdx.x, p.nitems, gridDim.x, p.ycols, p.zc, p.nz);
    TaskIter pf = it;  // load cursor: two tasks ahead of `it` after the prologue
    int issued = 0;    // loads issued so far (uniform)
    for (int k = 0; k < 2 && pf.valid(); ++k) {
        if (threadIdx.x == 0) issue_plane<VX>(in, p, pf.col, pf.pz, stg + k * G::STAGE, &bars[k]);
        ++issued;
        pf.next();
    }

    // accumulators: [0] plane behind, [1] current plane, [2] plane ahead
    float acc[3][VX][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < VX; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][i][c] = 0.f;

    for (int tc = 0; it.valid(); ++tc) {
        const int s = tc & 1;
        const float *stage = stg + s * G::STAGE;
        float *xbuf = xs + s * G::XBUF;
        const bool ok = mbar_wait(&bars[s], (uint32_t)((tc >> 1) & 1));
        const int mode = it.mode();
        if (ok) {
            if (mode == MID)
                phase_a<VX, MID, 0, 1, 2>(acc, stage, xbuf, p, lane, warp);
            else if (mode == FIRST)
                phase_a<VX, FIRST, 0, 1, 2>(acc, stage, xbuf, p, lane, warp);
            else
                phase_a<VX, LAST, 0, 1, 2>(acc, stage, xbuf, p, lane, warp);
        }
        if (!ok) failed = 1;  // a wait that gave up, seen by every thread after the barrier
        __syncthreads();
        if (failed) {
            // a copy never arrived: flag it, let the copies in flight land, stop
            if (threadIdx.x == 0) {
                atomicExch(p.err, 1);
                for (int t = tc + 1; t < issued; ++t) mbar_wait(&bars[t & 1], (uint32_t)((t >> 1) & 1));
            }
            return;
        }
        // every warp has consumed this stage: refill it two tasks ahead
        if (pf.valid()) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_plane<VX>(in, p, pf.col, pf.pz, stg + s * G::STAGE, &bars[s]);
            }
            ++issued;
            pf.next();
        }
        if (mode == MID) {
            phase_b<VX, MID, 0, 1, 2>(acc, xbuf, out, p, lane, warp, it.col,
                                      it.pz > it.za ? it.pz - 1 : -1);
            rotate(acc);
        } else if (mode == FIRST) {
            phase_b<VX, FIRST, 0, 1, 2>(acc, xbuf, out, p, lane, warp, it.col, -1);
            rotate(acc);  // plane za becomes the current plane
        } else {
            // LAST: the plane behind (zb - 1) completes the run; clear the plane
            // ahead's partial sums before the next run
            phase_b<VX, LAST, 0, 1, 2>(acc, xbuf, out, p, lane, warp, it.col, it.zb - 1);
#pragma unroll
            for (int a = 1; a < 3; ++a)
#pragma unroll
                for (int i = 0; i < VX; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][i][c] = 0.f;
        }
        it.next();
    }
}

template <int VX>
static cudaError_t prepare_vx(int *ctas) {
    static DevSlots slots;
    const int n = per_device(slots, [] {
        if (cudaFuncSetAttribute(k_d3q19_tiled<VX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Geo<VX>::BYTES) != cudaSuccess)
            return -1;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_d3q19_tiled<VX>, NTHREADS, Geo<VX>::BYTES) !=
                cudaSuccess ||
            nb < 1)
            return -1;
        return nb * device_sms();
    });
    if (ctas) *ctas = n;
    return n > 0 ? cudaSuccess : cudaErrorNotSupported;
}

// Planes per chunk: minimise the per-CTA critical path, i.e. the number of items
// per CTA times (planes per chunk + the two z-halo planes at about 0.35 of a
// plane each), over chunks of 4 .. nz planes.
int chunk_planes(int ycols, int nz, int ctas) {
    if (ctas < 1) ctas = 1;
    int best = nz;
    double best_t = 1e300;
    for (int zc = (nz < 4 ? nz : 4); zc <= nz; ++zc) {
        const long long items = (long long)ycols * ((nz + zc - 1) / zc);
        const long long per = (items + ctas - 1) / ctas;
        const double t = (double)per * (zc + 0.7);
        if (t < best_t - 1e-9) {
            best_t = t;
            best = zc;
        }
    }
    return best;
}

}  // namespace

bool tiled_supported(int Q, int storage, const StepParams &p) {
    if (Q != 19 || storage != STORE_F32) return false;
    // walled domains (cavity, channel): the kernel wraps every axis and the wall pass
    // after it recomputes every boundary node, the only nodes with a source outside
    if (p.has_force || p.gfield || p.sdelta != 0.f || p.scalar || p.bulk) return false;  // plain scheme only
    if (!(p.nx == 128 || p.nx == 256)) return false;
    if (p.ny % ROWS != 0 || p.ny < ROWS) return false;
    if (p.nz < 1) return false;
    if (p.fstride % 4 != 0) return false;  // 16-byte rows for the bulk copies
    if (!p.err) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return (p.nx == 256 ? prepare_vx<8>(nullptr) : prepare_vx<4>(nullptr)) == cudaSuccess;
}

template <int VX>
static cudaError_t launch_vx(const void *in, void *out, const StepParams &sp, cudaStream_t st) {
    int ctas = 0;
    cudaError_t e = prepare_vx<VX>(&ctas);
    if (e != cudaSuccess) return e;
    TiledParams p;
    p.nx = sp.nx;
    p.ny = sp.ny;
    p.nz = sp.nz;
    p.ycols = sp.ny / ROWS;
    p.zc = chunk_planes(p.ycols, sp.nz, ctas);
    p.nitems = p.ycols * ((sp.nz + p.zc - 1) / p.zc);
    p.fstride = sp.fstride;
    const double nu = (double)sp.s / 18.0;
    p.s18 = (float)nu;
    p.c4 = (float)(1.0 / (4.0 * nu));
    p.a_s = (float)((double)sp.a / nu);
    p.err = sp.err;
    const int grid = ctas < p.nitems ? ctas : p.nitems;
    k_d3q19_tiled<VX><<<(unsigned)grid, NTHREADS, Geo<VX>::BYTES, st>>>((const float *)in, (float *)out, p);
    return cudaGetLastError();
}

cudaError_t launch_step_tiled(int Q, int storage, const void *in, void *out, const StepParams &p,
                              cudaStream_t st) {
    if (!tiled_supported(Q, storage, p)) return cudaErrorNotSupported;
    if (p.nx == 256) return launch_vx<8>(in, out, p, st);
    return launch_vx<4>(in, out, p, st);
}

const char *tiled_name(int Q) { return Q == 9 ? "tiled_d2q9" : "tiled_d3q19_tma"; }

}  // namespace lwacm
