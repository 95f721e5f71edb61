// Building blocks shared by the row-tiled D3Q19 kernels (kernels_tiled.cu,
// kernels_half.cu): per-launch parameters, mbarrier / bulk-copy wrappers, the
// task iterator over (y-column, z-chunk) work items, the link-value arithmetic of
// the moment form (lwacm_core.cuh) and lane-row shifts and shared-memory slots.
#pragma once

#include <stdint.h>
#include <string.h>

#include "lwacm_core.cuh"

namespace lwacm {
namespace tile {

constexpr int ROWS = 8;
constexpr int TROWS = ROWS + 2;  // staged rows: y0-1, y0 .. y0+7, y0+8
constexpr int NSLOT = 4;         // values passed per receiver and direction
constexpr unsigned FULL = 0xffffffffu;

struct TiledParams {
    int nx, ny, nz;
    int ycols;           // ny / ROWS
    int zc, nitems;      // planes per chunk, ycols * ceil(nz / zc)
    long long fstride;
    float s18;           // s / 18 = nu
    float c4;            // 1 / (4 nu)
    float a_s;           // a / nu
    int *err;            // error word (timeout)
};

// ---- PTX wrappers: mbarrier and 1-D bulk copy ---------------------------------
__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: at most 2^22 polls with back-off (well under a second)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_test(bar, parity)) return true;
        if (it > 32) __nanosleep(100);
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            sa(dst)),
        "l"(src), "r"(bytes), "r"(sa(bar))
        : "memory");
}

// 1/x: hardware approximation refined by one Newton-Raphson step
// (r <- r + r (1 - x r)), accurate to about an ulp for the densities here.
__device__ __forceinline__ float rcp_nr(float x) {
    float r = __fdividef(1.0f, x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// ---- task iteration -------------------------------------------------------------
// Work items are (column, z-chunk) pairs, numbered chunk-major (item = chunk * ycols
// + col) so that the CTAs working on neighbouring columns march through the same
// planes together and share their halo rows in L2. CTA b takes items b, b + G,
// b + 2G, ... (G = grid size). An item is a run [za, zb) of planes of one column,
// processed as source planes za-1 (FIRST), za .. zb-1 (MID), zb (LAST).
enum { FIRST = 0, MID = 1, LAST = 2 };

struct TaskIter {
    int item, nitems, stride, ycols, zc, nz;
    int col, za, zb, pz;
    __device__ void start_run() {
        col = item % ycols;
        const int ch = item / ycols;
        za = ch * zc;
        zb = za + zc < nz ? za + zc : nz;
        pz = za - 1;
    }
    __device__ TaskIter(int first, int nitems_, int stride_, int ycols_, int zc_, int nz_)
        : item(first), nitems(nitems_), stride(stride_), ycols(ycols_), zc(zc_), nz(nz_) {
        col = za = zb = pz = 0;
        if (item < nitems) start_run();
    }
    __device__ bool valid() const { return item < nitems; }
    __device__ int mode() const { return pz < za ? FIRST : (pz < zb ? MID : LAST); }
    __device__ void next() {
        if (pz < zb) {
            ++pz;
        } else {
            item += stride;
            if (item < nitems) start_run();
        }
    }
};

// position of node group h (4 nodes) of lane l inside an exchange row: the 4-float
// groups of all lanes are contiguous, so warp float4 accesses are conflict-free
__device__ __forceinline__ int spos(int l, int h) { return h * 128 + l * 4; }

// deposit the value g of link c = (cx,cy,cz) into a receiver's (d, jx, jy, jz).
// Values arriving along c_z = +1 links feed the plane ahead, which receives
// nothing else before it becomes the current plane; its jz then equals its d and
// is copied at that point, so those deposits skip jz.
__device__ __forceinline__ void dep(float (&a)[4], float g, int cx, int cy, int cz) {
    a[0] += g;
    if (cx > 0) a[1] += g;
    if (cx < 0) a[1] -= g;
    if (cy > 0) a[2] += g;
    if (cy < 0) a[2] -= g;
    if (cz < 0) a[3] -= g;
}

template <int PM, int P0, int PP>
__device__ __forceinline__ constexpr int pl(int cz) { return cz > 0 ? PP : (cz < 0 ? PM : P0); }

// per-node constants: velocity and, with K = d - 3/2 rho |u|^2, the three
// coefficients of a link value w [d + rho (s e + 9/2 e^2 - 3/2 |u|^2)] =
// w K + w rho s e + w 9/2 rho e^2 (e = c.u) for the axis weight w = 1/18
// (K1 = K/18, A1 = rho s/18 = rho nu, B1 = rho/4) and the diagonal weight
// 1/36 (K2, A2, B2: half of those).
template <int VX>
struct NodeConst {
    float U[VX], V[VX], W[VX], K1[VX], A1[VX], B1[VX], K2[VX], A2[VX], B2[VX];
};

// four consecutive stored values as floats (FP32, or BF16 / FP16 storage: a
// bfloat16 is the upper half of an FP32, so widening it is exact)
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p) {
    const uint2 r = *reinterpret_cast<const uint2 *>(p);
    return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u),
                       __uint_as_float(r.y << 16), __uint_as_float(r.y & 0xffff0000u));
}
__device__ __forceinline__ float4 ld4(const __half *p) {
    const uint2 r = *reinterpret_cast<const uint2 *>(p);
    __half2 a, b;
    memcpy(&a, &r.x, 4);
    memcpy(&b, &r.y, 4);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
// store four floats rounded (to nearest even) to the storage type
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(__nv_bfloat16 *p, float a, float b, float c, float d) {
    const __nv_bfloat162 x = __floats2bfloat162_rn(a, b), y = __floats2bfloat162_rn(c, d);
    uint2 r;
    memcpy(&r.x, &x, 4);
    memcpy(&r.y, &y, 4);
    *reinterpret_cast<uint2 *>(p) = r;
}
__device__ __forceinline__ void st4(__half *p, float a, float b, float c, float d) {
    const __half2 x = __floats2half2_rn(a, b), y = __floats2half2_rn(c, d);
    uint2 r;
    memcpy(&r.x, &x, 4);
    memcpy(&r.y, &y, 4);
    *reinterpret_cast<uint2 *>(p) = r;
}

// row: staged field-0 row; rstride: distance (in elements) between fields in the stage
template <int VX, typename T>
__device__ __forceinline__ void node_consts(NodeConst<VX> &nc, const T *row, int rstride, int lane,
                                            float s18) {
#pragma unroll
    for (int h = 0; h < VX / 4; ++h) {
        const float4 d4 = ld4(row + lane * VX + 4 * h);
        const float4 u4 = ld4(row + rstride + lane * VX + 4 * h);
        const float4 v4 = ld4(row + 2 * rstride + lane * VX + 4 * h);
        const float4 w4 = ld4(row + 3 * rstride + lane * VX + 4 * h);
        const float dd[4] = {d4.x, d4.y, d4.z, d4.w}, uu[4] = {u4.x, u4.y, u4.z, u4.w};
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w}, ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = 4 * h + j;
            const float rho = 1.f + dd[j];
            const float q = fmaf(uu[j], uu[j], fmaf(vv[j], vv[j], ww[j] * ww[j]));
            const float K = fmaf(-1.5f * rho, q, dd[j]);
            nc.U[i] = uu[j];
            nc.V[i] = vv[j];
            nc.W[i] = ww[j];
            nc.K1[i] = K * (1.f / 18.f);
            nc.A1[i] = rho * s18;
            nc.B1[i] = 0.25f * rho;
            nc.K2[i] = K * (1.f / 36.f);
            nc.A2[i] = rho * (0.5f * s18);
            nc.B2[i] = 0.125f * rho;
        }
    }
}

// values of the pair (c, -c) at node i (e = c.u): the even part w (K + 9/2 rho e^2)
// plus or minus the odd part w rho s e; axis links weight 1/18, diagonals 1/36
template <int VX>
__device__ __forceinline__ void pair_g(const NodeConst<VX> &nc, int i, float e, bool diag, float &gp,
                                       float &gm) {
    const float A = diag ? nc.A2[i] : nc.A1[i];
    const float cm = fmaf((diag ? nc.B2[i] : nc.B1[i]) * e, e, diag ? nc.K2[i] : nc.K1[i]);
    gp = fmaf(A, e, cm);
    gm = fmaf(-A, e, cm);
}

// the five (c, -c) pairs with c_y(c) = +1: c = (cx, 1, cz)
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

}  // namespace tile
}  // namespace lwacm
