// Register-prefetch z-marching kernel for D3Q19 on periodic domains with nx = 32*VX (VX = 4, 8),
// ny a multiple of 8: the moment form of Eq. ACM2.0 (see lwacm_core.cuh) with
// every field read from HBM once and written once per step.
//
// CTA = 8 row warps. Row warp w owns the full x-row y0 + w of the
// current z-plane, lane l the VX consecutive nodes x = l*VX .. l*VX+VX-1, so the
// periodic x-neighbours of a row are reached with warp shuffles (lane 31 wraps to
// lane 0). The CTA marches along z through its chunk [z0, z1); per plane each
// node computes its 19 outgoing values g_i once (pre-combine, Eq. ACM2.0b(a)) and
// they are streamed (Eq. ACM2.0b(b)) to their receivers:
//   * links with c_y = 0 stay in the warp: register moves, one shuffle per link
//     at lane boundaries;
//   * links with c_y = +-1 go through shared memory to the warp of the next /
//     previous row (double-buffered, one barrier per plane); warps 0 and 7 also
//     compute the c_y = +1 values of row y0-1 and the c_y = -1 values of row y0+8;
//   * links with c_z = +-1 land in the accumulators of planes z+-1, which live in
//     registers: three planes of (d, jx, jy, jz) rotate as the CTA marches.
// Plane z-1 is complete once plane z has been processed; it is post-combined
// (Eq. ACM2.0b(c): + a rho u), divided by rho (moments, Section 2.1) and stored.
// The next plane's fields are loaded into registers while the current plane's
// exchange and stores proceed.
#include "dev_cache.h"
#include "launch.h"
#include "lwacm_core.cuh"

namespace lwacm {
namespace zm {

constexpr int ROWS = 8;
constexpr int NWARPS = ROWS;  // warps 0 and ROWS-1 also compute the halo rows
constexpr int NTHREADS = NWARPS * 32;
constexpr unsigned FULL = 0xffffffffu;

struct TiledParams {
    int nx, ny, nz, zc;
    long long fstride;
    float s18;   // s / 18 = nu
    float c4;    // 1 / (4 nu): turns rho nu e into the rho e / 4 of the 9/2 (c.u)^2 term
    float a_s;   // a / nu: turns rho nu into a rho
};

template <int VX>
struct Geo {
    static constexpr int RL = 32 * VX;        // row length in floats
    static constexpr int SLOT = ROWS * RL;     // one link slot, all receiver rows
    static constexpr int DIR = 5 * SLOT;       // five links per direction
    static constexpr int BUF = 2 * DIR;        // up + down
    static constexpr size_t BYTES = 2 * BUF * sizeof(float);  // double-buffered
};

// position of node i of lane l inside a row slot: 4-float groups of all lanes
// are contiguous, so float4 accesses of a warp are bank-conflict free
__device__ __forceinline__ int spos(int l, int h) { return h * 128 + l * 4; }

template <int VX>
__device__ __forceinline__ void load_plane(float (&F)[4][VX], const float *__restrict__ base,
                                           long long fstride) {
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int h = 0; h < VX / 4; ++h) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(base + f * fstride) + h);
            F[f][4 * h + 0] = t.x;
            F[f][4 * h + 1] = t.y;
            F[f][4 * h + 2] = t.z;
            F[f][4 * h + 3] = t.w;
        }
}

// deposit the value g of link c = (cx,cy,cz) into a receiver's (d, jx, jy, jz).
// Links with c_z = +1 feed the plane ahead, which receives nothing else before it
// becomes the current plane: its jz equals its d then and is copied at that
// point, so those deposits skip jz.
__device__ __forceinline__ void dep(float (&a)[4], float g, int cx, int cy, int cz) {
    a[0] += g;
    if (cx > 0) a[1] += g;
    if (cx < 0) a[1] -= g;
    if (cy > 0) a[2] += g;
    if (cy < 0) a[2] -= g;
    if (cz < 0) a[3] -= g;
}

// plane slot for a link with z-component cz, given the rotating indices
template <int PM, int P0, int PP>
__device__ __forceinline__ constexpr int pl(int cz) { return cz > 0 ? PP : (cz < 0 ? PM : P0); }

// The five (c, -c) pairs whose c has c_y = +1; c = (cx, 1, cz), diag = |c|^2 == 2.
__device__ __forceinline__ constexpr int ypair_cx(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
__device__ __forceinline__ constexpr int ypair_cz(int k) { return k == 3 ? 1 : (k == 4 ? -1 : 0); }

// per-node constants: velocity, K/18 with K = d - 3/2 rho |u|^2, and rho nu
// (= rho s / 18). A link value is then w/(1/18) * (K1 + A1 e (1 + e / (4 nu)))
// = w [d + rho (s e + 9/2 e^2 - 3/2 |u|^2)] with e = c.u.
template <int VX>
struct NodeConst {
    float U[VX], V[VX], W[VX], K1[VX], A1[VX];
};

template <int VX>
__device__ __forceinline__ void node_consts(NodeConst<VX> &nc, const float (&F)[4][VX], float s18) {
#pragma unroll
    for (int i = 0; i < VX; ++i) {
        const float d = F[0][i], u = F[1][i], v = F[2][i], w = F[3][i];
        const float rho = 1.f + d;
        const float q = fmaf(u, u, fmaf(v, v, w * w));
        const float K = fmaf(-1.5f * rho, q, d);  // d - 3/2 rho |u|^2
        nc.U[i] = u;
        nc.V[i] = v;
        nc.W[i] = w;
        nc.K1[i] = K * (1.f / 18.f);
        nc.A1[i] = rho * s18;  // rho s / 18
    }
}

// g for the pair (c, -c) at node i: axis links weight 1/18, diagonals 1/36
template <int VX>
__device__ __forceinline__ void pair_g(const NodeConst<VX> &nc, int i, float e, bool diag,
                                       float c4, float &gp, float &gm) {
    const float od = nc.A1[i] * e;                // rho s e / 18
    const float cm = fmaf(od * c4, e, nc.K1[i]);  // (K + 9/2 rho e^2) / 18
    if (diag) {
        const float ho = 0.5f * od;
        gp = fmaf(0.5f, cm, ho);
        gm = fmaf(0.5f, cm, -ho);
    } else {
        gp = cm + od;
        gm = cm - od;
    }
}

template <int VX>
__device__ __forceinline__ float ypair_e(const NodeConst<VX> &nc, int k, int i) {
    const float u = nc.U[i], v = nc.V[i], w = nc.W[i];
    return k == 0 ? v : (k == 1 ? u + v : (k == 2 ? v - u : (k == 3 ? v + w : v - w)));
}

// shift a lane-distributed row in place by +1 (g[x] <- g[x-1]) or -1 (g[x] <- g[x+1])
template <int VX>
__device__ __forceinline__ void xshift(float (&g)[VX], int dir, int lane) {
    if (dir > 0) {
        const float e = __shfl_sync(FULL, g[VX - 1], (lane + 31) & 31);
#pragma unroll
        for (int i = VX - 1; i > 0; --i) g[i] = g[i - 1];
        g[0] = e;
    } else if (dir < 0) {
        const float e = __shfl_sync(FULL, g[0], (lane + 1) & 31);
#pragma unroll
        for (int i = 0; i < VX - 1; ++i) g[i] = g[i + 1];
        g[VX - 1] = e;
    }
}

template <int VX>
__device__ __forceinline__ void st_slot(float *slot, const float (&o)[VX], int lane) {
#pragma unroll
    for (int h = 0; h < VX / 4; ++h)
        *reinterpret_cast<float4 *>(slot + spos(lane, h)) =
            make_float4(o[4 * h], o[4 * h + 1], o[4 * h + 2], o[4 * h + 3]);
}

template <int VX>
__device__ __forceinline__ void ld_slot(const float *slot, float (&o)[VX], int lane) {
#pragma unroll
    for (int h = 0; h < VX / 4; ++h) {
        const float4 t = *reinterpret_cast<const float4 *>(slot + spos(lane, h));
        o[4 * h] = t.x;
        o[4 * h + 1] = t.y;
        o[4 * h + 2] = t.z;
        o[4 * h + 3] = t.w;
    }
}

template <int VX, int PM, int P0, int PP>
__device__ __forceinline__ void plane_step(float (&acc)[3][VX][4], float (&F)[4][VX],
                                           float (&Fh)[4][VX], int pz, int z0, int z1,
                                           const TiledParams &p, int lane, int warp, int yrow,
                                           int hrow, const float *__restrict__ in,
                                           float *__restrict__ out, float *xs) {
    using G = Geo<VX>;
    float *buf = xs + (pz & 1) * G::BUF;  // pz may be -1: & 1 still alternates
    float *up = buf, *dn = buf + G::DIR;
    const long long rowoff = (long long)yrow * p.nx + lane * VX;
    const long long hrowoff = (long long)hrow * p.nx + lane * VX;
    const long long plane = (long long)p.nx * p.ny;

    {
        NodeConst<VX> nc;
        node_consts(nc, F, p.s18);
        // ---- rest link, post-combine term a rho u, z-links -------------------
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            // the receiver plane's z-momentum so far equals its density sum: every
            // value it received came along a c_z = +1 link (see plane rotation)
            acc[P0][i][3] = acc[P0][i][0];
            acc[P0][i][0] += 6.f * nc.K1[i];  // w_0 K = K/3
            const float ar = p.a_s * nc.A1[i];  // a rho
            acc[P0][i][1] = fmaf(ar, nc.U[i], acc[P0][i][1]);
            acc[P0][i][2] = fmaf(ar, nc.V[i], acc[P0][i][2]);
            acc[P0][i][3] = fmaf(ar, nc.W[i], acc[P0][i][3]);
            float gp, gm;
            pair_g(nc, i, nc.W[i], false, p.c4, gp, gm);  // (0,0,+1) / (0,0,-1)
            acc[PP][i][0] += gp;  // c = (0,0,+1): jz of plane PP is implied by d
            dep(acc[PM][i], gm, 0, 0, -1);
        }
        // ---- in-row links c = (1,0,cz) / -c --------------------------------
#pragma unroll
        for (int cz = -1; cz <= 1; ++cz) {
            float eP = 0.f, eM = 0.f;
#pragma unroll
            for (int i = 0; i < VX; ++i) {
                float gp, gm;
                const float e = cz == 0 ? nc.U[i] : (cz > 0 ? nc.U[i] + nc.W[i] : nc.U[i] - nc.W[i]);
                pair_g(nc, i, e, cz != 0, p.c4, gp, gm);
                if (i + 1 < VX)
                    dep(acc[pl<PM, P0, PP>(cz)][i + 1], gp, 1, 0, cz);
                else
                    eP = gp;
                if (i > 0)
                    dep(acc[pl<PM, P0, PP>(-cz)][i - 1], gm, -1, 0, -cz);
                else
                    eM = gm;
            }
            const float rP = __shfl_sync(FULL, eP, (lane + 31) & 31);
            const float rM = __shfl_sync(FULL, eM, (lane + 1) & 31);
            dep(acc[pl<PM, P0, PP>(cz)][0], rP, 1, 0, cz);
            dep(acc[pl<PM, P0, PP>(-cz)][VX - 1], rM, -1, 0, -cz);
        }
        // ---- row-crossing links: to shared memory ---------------------------
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float gp[VX], gm[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) pair_g(nc, i, ypair_e(nc, k, i), k != 0, p.c4, gp[i], gm[i]);
            if (warp + 1 < ROWS) {  // c (c_y = +1) to the next row, receiver x <- source x - cx
                xshift(gp, ypair_cx(k), lane);
                st_slot(up + k * G::SLOT + (warp + 1) * G::RL, gp, lane);
            }
            if (warp > 0) {  // -c (c_y = -1) to the previous row, receiver x <- source x + cx
                xshift(gm, -ypair_cx(k), lane);
                st_slot(dn + k * G::SLOT + (warp - 1) * G::RL, gm, lane);
            }
        }
    }
    // ---- halo rows: bottom (y0-1) feeds row 0, top (y0+ROWS) feeds row ROWS-1 --
    if (warp == 0 || warp == ROWS - 1) {
        NodeConst<VX> hc;
        node_consts(hc, Fh, p.s18);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float gp[VX], gm[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) pair_g(hc, i, ypair_e(hc, k, i), k != 0, p.c4, gp[i], gm[i]);
            if (warp == 0) {  // c_y = +1 values of row y0-1
                xshift(gp, ypair_cx(k), lane);
                st_slot(up + k * G::SLOT, gp, lane);
            } else {  // c_y = -1 values of row y0+ROWS
                xshift(gm, -ypair_cx(k), lane);
                st_slot(dn + k * G::SLOT + (ROWS - 1) * G::RL, gm, lane);
            }
        }
    }

    // ---- prefetch the next plane while the exchange completes -------------
    if (pz + 1 <= z1) {
        int zn = pz + 1;
        zn = zn >= p.nz ? zn - p.nz : zn;
        load_plane<VX>(F, in + (long long)zn * plane + rowoff, p.fstride);
        if (warp == 0 || warp == ROWS - 1)
            load_plane<VX>(Fh, in + (long long)zn * plane + hrowoff, p.fstride);
    }
    __syncthreads();

    {
        // ---- receive row-crossing links ---------------------------------------
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float o[VX];
            const int cx = ypair_cx(k), cz = ypair_cz(k);
            ld_slot(up + k * G::SLOT + warp * G::RL, o, lane);
#pragma unroll
            for (int i = 0; i < VX; ++i) dep(acc[pl<PM, P0, PP>(cz)][i], o[i], cx, 1, cz);
            ld_slot(dn + k * G::SLOT + warp * G::RL, o, lane);
#pragma unroll
            for (int i = 0; i < VX; ++i) dep(acc[pl<PM, P0, PP>(-cz)][i], o[i], -cx, -1, -cz);
        }
        // ---- plane pz-1 is complete: moments, store, reset ---------------------
        const int zr = pz - 1;
        if (zr >= z0 && zr < z1) {
            float *o = out + (long long)zr * plane + rowoff;
            float r[VX];
#pragma unroll
            for (int i = 0; i < VX; ++i) r[i] = __frcp_rn(1.f + acc[PM][i][0]);
#pragma unroll
            for (int h = 0; h < VX / 4; ++h) {
#define LW_ST(F, C, SC)                                                                          \
    reinterpret_cast<float4 *>(o + (F) * p.fstride)[h] =                                         \
        make_float4(acc[PM][4 * h][C] * (SC ? r[4 * h] : 1.f),                                   \
                    acc[PM][4 * h + 1][C] * (SC ? r[4 * h + 1] : 1.f),                           \
                    acc[PM][4 * h + 2][C] * (SC ? r[4 * h + 2] : 1.f),                           \
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

// 8 warps: up to 255 registers per thread; launch_vx checks the occupancy
// before the first launch.
template <int VX>
__global__ void __launch_bounds__(NTHREADS, 1) k_d3q19_zmarch(const float *__restrict__ in, float *__restrict__ out, TiledParams p) {
    extern __shared__ float4 smem4[];
    float *xs = reinterpret_cast<float *>(smem4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int y0 = blockIdx.x * ROWS;
    const int z0 = blockIdx.y * p.zc;
    const int z1 = min(z0 + p.zc, p.nz);
    const int yrow = y0 + warp;
    // halo row of warps 0 / ROWS-1 (periodic in y); unused by the other warps
    int hrow = warp == 0 ? y0 - 1 : y0 + ROWS;
    hrow = hrow < 0 ? hrow + p.ny : (hrow >= p.ny ? hrow - p.ny : hrow);
    const long long plane = (long long)p.nx * p.ny;
    const long long rowoff = (long long)yrow * p.nx + lane * VX;
    const long long hrowoff = (long long)hrow * p.nx + lane * VX;

    float acc[3][VX][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < VX; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][i][c] = 0.f;
    float F[4][VX], Fh[4][VX];
    {
        int zs = z0 - 1;
        zs = zs < 0 ? zs + p.nz : zs;
        load_plane<VX>(F, in + (long long)zs * plane + rowoff, p.fstride);
        if (warp == 0 || warp == ROWS - 1)
            load_plane<VX>(Fh, in + (long long)zs * plane + hrowoff, p.fstride);
    }
    // source planes z0-1 .. z1; receiver plane pz-1 completes at source plane pz
    for (int pz = z0 - 1; pz <= z1; pz += 3) {
        plane_step<VX, 0, 1, 2>(acc, F, Fh, pz, z0, z1, p, lane, warp, yrow, hrow, in, out, xs);
        if (pz + 1 <= z1)
            plane_step<VX, 1, 2, 0>(acc, F, Fh, pz + 1, z0, z1, p, lane, warp, yrow, hrow, in, out, xs);
        if (pz + 2 <= z1)
            plane_step<VX, 2, 0, 1>(acc, F, Fh, pz + 2, z0, z1, p, lane, warp, yrow, hrow, in, out, xs);
    }
}

int chunk_for(const StepParams &p) {
    // CTAs = (ny/8) x ceil(nz/zc): aim for a whole number of waves at one CTA
    // per SM with chunks of >= 8 planes.
    const int sms = device_sms();
    const int ycta = p.ny / ROWS;
    int best = p.nz, best_score = -1;
    for (int zc = 8; zc <= p.nz; ++zc) {
        const int nch = (p.nz + zc - 1) / zc;
        const long long ctas = (long long)ycta * nch;
        const long long waves = (ctas + sms - 1) / sms;
        // efficiency: useful work / (waves * sms * zc) with a 2-plane halo cost
        const double eff = (double)ycta * p.nz / ((double)waves * sms * (zc + 0.6));
        const int score = (int)(eff * 1e6);
        if (score > best_score) {
            best_score = score;
            best = zc;
        }
    }
    return best;
}

// One-time set-up per kernel instance: opt in to the shared-memory size and
// check that one CTA fits on an SM (registers + shared memory).
template <int VX>
static cudaError_t prepare_vx() {
    static DevSlots slots;  // per device: 1 ok, -1 does not fit
    const int state = per_device(slots, [] {
        if (cudaFuncSetAttribute(k_d3q19_zmarch<VX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Geo<VX>::BYTES) != cudaSuccess)
            return -1;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_d3q19_zmarch<VX>, NTHREADS, Geo<VX>::BYTES) !=
            cudaSuccess)
            return -1;
        return nb >= 1 ? 1 : -1;
    });
    return state == 1 ? cudaSuccess : cudaErrorNotSupported;
}

}  // namespace zm

using namespace zm;

bool zmarch_supported(int Q, int storage, const StepParams &p) {
    if (Q != 19 || storage != STORE_F32) return false;
    // walled domains (cavity, channel): the kernel wraps every axis and the wall pass
    // after it recomputes every boundary node, the only nodes with a source outside
    if (p.has_force || p.gfield || p.sdelta != 0.f || p.scalar || p.bulk) return false;  // plain scheme only
    if (!(p.nx == 128 || p.nx == 256)) return false;
    if (p.ny % ROWS != 0 || p.ny < ROWS) return false;
    if (p.nz < 1) return false;
    if (p.fstride % 4 != 0) return false;  // float4 rows
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;  // no device: cannot run it anyway
    return (p.nx == 256 ? prepare_vx<8>() : prepare_vx<4>()) == cudaSuccess;
}

template <int VX>
static cudaError_t launch_vx(const void *in, void *out, const StepParams &sp, cudaStream_t st) {
    cudaError_t e = prepare_vx<VX>();
    if (e != cudaSuccess) return e;
    TiledParams p;
    p.nx = sp.nx;
    p.ny = sp.ny;
    p.nz = sp.nz;
    p.fstride = sp.fstride;
    const double nu = (double)sp.s / 18.0;
    p.s18 = (float)nu;
    p.c4 = (float)(1.0 / (4.0 * nu));
    p.a_s = (float)((double)sp.a / nu);
    p.zc = chunk_for(sp);
    dim3 grid(sp.ny / ROWS, (sp.nz + p.zc - 1) / p.zc);
    k_d3q19_zmarch<VX><<<grid, NTHREADS, Geo<VX>::BYTES, st>>>((const float *)in, (float *)out, p);
    return cudaGetLastError();
}

cudaError_t launch_step_zmarch(int Q, int storage, const void *in, void *out, const StepParams &p,
                               cudaStream_t st) {
    if (!zmarch_supported(Q, storage, p)) return cudaErrorNotSupported;
    if (p.nx == 256) return launch_vx<8>(in, out, p, st);
    return launch_vx<4>(in, out, p, st);
}


}  // namespace lwacm
