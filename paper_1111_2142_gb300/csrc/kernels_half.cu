// Half-row TMA row-tiled D3Q19 kernel, for domains with nx = 256, 128 or other rows
// of at least 72 nodes (multiples of 4, see segments_fit) and any ny (periodic; walled domains get the wall pass after it,
// the cavity's x faces handled here for rows of 128 and 256): the moment form of
// Eq. ACM2.0 (see lwacm_core.cuh), every field read from HBM once and written once
// per step. A CTA updates columns of 8 rows; when ny % 8 != 0 the last column's
// rows beyond ny hold the rows that follow it periodically, so its first such row
// feeds the last real row from above as a halo row would, and none of them is stored.
//
// Persistent CTAs over (y-column, run of planes) items, scheduled as equal runs or
// z-chunks (TaskIter and plan_schedule in tile_common.cuh), TMA bulk copies of ten
// staged rows per plane, packed row exchange through shared memory, three rotating
// accumulator planes; each 256-node row is shared by two warps (half h covers
// x = 128 h .. 128 h + 127, four nodes per lane), so a CTA of 8 rows has 16 warps
// at up to 128 registers per thread.
//
// The two halves of a row meet at x = 127|128 and, periodically, at x = 255|0. A
// shuffle cannot cross them, so each half's boundary lanes (0 and 31) recompute
// the link values they take from their neighbour node in the other half (in-row
// links and the x-shifted row-crossing diagonals) from that node's staged fields:
// the halves exchange nothing.
//
// nx = 128 uses the same code with one warp per row (NH = 1): the warp's shuffles
// wrap x periodically by themselves, and two CTAs of 8 warps share an SM. Longer
// rows (NH = 0) are cut into 128-node segments, one warp each, whose boundary lanes
// recompute their outside neighbours' link values like the halves do, from 8 extra
// staged nodes on each side.
#include <stdint.h>

#include "dev_cache.h"
#include "launch.h"
#include "lwacm_core.cuh"
#include "tile_common.cuh"

namespace lwacm {
namespace {

using namespace tile;

constexpr int VXH = 4;                 // nodes per lane
constexpr int HALF = 128;              // nodes per warp row segment
constexpr int HALF_ROWS = 8;           // rows per column of the 256-node-row form

// Row geometry. NH = 1: one warp per row of nx = 128 nodes, its lanes wrap
// periodically by themselves; NH = 2: two warps (halves) per row of 256, see above;
// NH = 0: other rows (nx >= 72) cut into ceil(nx / 128) segments of 128, one warp
// per segment and a CTA per (segment, column of rows): the staged rows carry 8 more
// nodes on each side (x0 - 8 .. x0 + 135, wrapped), and the boundary lanes take
// their outside neighbours from them as the halves do. A short last segment stages
// the row's first nodes after its end, and its lanes there store nothing.
template <int NH>
struct HGeo {
    static constexpr bool SEG = NH == 0;
    static constexpr int RW = NH == 2 ? HALF_ROWS : ROWS;  // rows of a column (a CTA's work item)
    static constexpr int TRW = RW + 2;              // staged rows: y0-1, y0 .. y0+RW-1, y0+RW
    static constexpr int NW = NH == 2 ? 2 : 1;      // warps per row (or segment)
    static constexpr int NTH = RW * NW * 32;        // threads per CTA
    static constexpr int MINB = NH == 2 && RW == 8 ? 1 : 2;  // CTAs per SM
    static constexpr int RL = HALF * NW;            // nodes of a row a CTA updates
    static constexpr int SRL = SEG ? HALF + 16 : RL;  // staged row length
    static constexpr int OWN = SEG ? 8 : 0;         // staged index of the first own node
    static constexpr bool NB = NH != 1;             // boundary lanes read their outside neighbours
    static constexpr int XSLOT = RW * RL;
    static constexpr int XDIR = NSLOT * XSLOT;
    static constexpr int XBUF = 2 * XDIR;  // floats
    // staged indices of the neighbours lane 0 (left) and lane 31 (right) of half h take
    __device__ static int left(int h) { return SEG ? OWN - 1 : (h * HALF + RL - 1) % RL; }
    __device__ static int right(int h) { return SEG ? OWN + HALF : (h * HALF + HALF) % RL; }
};
// T: storage type of the fields (FP32, or BF16 / FP16 widened to FP32 on load).
template <int NH, typename T = float>
struct HG : HGeo<NH> {
    static constexpr int STAGE = 4 * HGeo<NH>::TRW * HGeo<NH>::SRL;  // elements of T
    static constexpr size_t BYTES = 2 * (size_t)HGeo<NH>::XBUF * 4 + 2 * (size_t)STAGE * sizeof(T) + 64;
    static constexpr uint32_t TX = STAGE * sizeof(T);
};

// ---- packed arithmetic ----------------------------------------------------------
// The four nodes of a lane are held as two pairs, (0,1) and (2,3), in float2
// registers, so that the same operation on two nodes issues as one packed FP32x2
// instruction (half the issue slots of two scalar ones, same rounding).
using F2 = float2;
__device__ __forceinline__ F2 b2(float v) { return make_float2(v, v); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 neg2(F2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }

// Per-node constants of the moment form, per node pair: the velocity and, with
// K = d - 3/2 rho |u|^2, the three coefficients of a link value
// w [d + rho (s e + 9/2 e^2 - 3/2 |u|^2)] = w K + w rho s e + w 9/2 rho e^2 (e = c.u)
// for the axis weight w = 1/18 (K1 = K/18, A1 = rho s/18 = rho nu, B1 = rho/4) and
// the diagonal weight 1/36 (K2, A2, B2: half of those).
struct NC2 {
    F2 U[2], V[2], W[2], K1[2], A1[2], B1[2], K2[2], A2[2], B2[2];
    F2 M[2];  // a d - 6 nu: a rho u = u + M u (post_combine, lwacm_core.cuh)
    F2 D[2];  // d (the forced variant: rho g = g + d g)
};

template <typename T>
__device__ __forceinline__ void node_consts2(NC2 &nc, const T *row, int rstride, int lane, float s18,
                                             float a = 0.f, float am1 = 0.f) {
    const float4 d4 = ld4(row + lane * VXH), u4 = ld4(row + rstride + lane * VXH);
    const float4 v4 = ld4(row + 2 * rstride + lane * VXH), w4 = ld4(row + 3 * rstride + lane * VXH);
    const F2 dd[2] = {make_float2(d4.x, d4.y), make_float2(d4.z, d4.w)};
    nc.U[0] = make_float2(u4.x, u4.y);
    nc.U[1] = make_float2(u4.z, u4.w);
    nc.V[0] = make_float2(v4.x, v4.y);
    nc.V[1] = make_float2(v4.z, v4.w);
    nc.W[0] = make_float2(w4.x, w4.y);
    nc.W[1] = make_float2(w4.z, w4.w);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const F2 rho = add2(dd[j], b2(1.f));
        const F2 q = fma2(nc.U[j], nc.U[j], fma2(nc.V[j], nc.V[j], mul2(nc.W[j], nc.W[j])));
        const F2 K = fma2(mul2(b2(-1.5f), rho), q, dd[j]);  // d - 3/2 rho |u|^2
        nc.K1[j] = mul2(K, b2(1.f / 18.f));
        nc.A1[j] = mul2(rho, b2(s18));
        nc.B1[j] = mul2(rho, b2(0.25f));
        nc.K2[j] = mul2(K, b2(1.f / 36.f));
        nc.A2[j] = mul2(rho, b2(0.5f * s18));
        nc.B2[j] = mul2(rho, b2(0.125f));
        nc.M[j] = fma2(b2(a), dd[j], b2(am1));
        nc.D[j] = dd[j];
    }
}

// values of the link pair (c, -c) at the two nodes of pair j, e = c.u
__device__ __forceinline__ void pair2(const NC2 &nc, int j, F2 e, bool diag, F2 &gp, F2 &gm) {
    const F2 A = diag ? nc.A2[j] : nc.A1[j], B = diag ? nc.B2[j] : nc.B1[j], K = diag ? nc.K2[j] : nc.K1[j];
    // scalar on purpose: the same arithmetic as FP32x2 operations measured 3% slower
    // (the FMA pipe, not instruction issue, is what these values contend for)
    const float cx = fmaf(B.x * e.x, e.x, K.x), cy = fmaf(B.y * e.y, e.y, K.y);
    gp = make_float2(fmaf(A.x, e.x, cx), fmaf(A.y, e.y, cy));
    gm = make_float2(fmaf(-A.x, e.x, cx), fmaf(-A.y, e.y, cy));
}

// The boundary neighbour of a half row (NH = 2): lanes 0-15 take node x0 - 1 (the
// one lane 0 receives from), lanes 16-31 node x0 + 128 (lane 31's), both wrapped
// periodically. sA = +A for lanes 0-15 and -A for lanes 16-31, so that one value
// c + sA e serves lane 0 (the link towards +x) and lane 31 (towards -x).
struct NbC {
    float U, V, W, K1, sA1, B1, K2, sA2, B2;
};
__device__ __forceinline__ float ld1(const float *p) { return *p; }
__device__ __forceinline__ float ld1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld1(const __half *p) { return __half2float(*p); }

template <typename T>
__device__ __forceinline__ NbC nb_consts(const T *row, int rstride, int nbx, float sgn, float s18) {
    NbC c;
    const float d = ld1(row + nbx);
    c.U = ld1(row + rstride + nbx);
    c.V = ld1(row + 2 * rstride + nbx);
    c.W = ld1(row + 3 * rstride + nbx);
    const float rho = 1.f + d;
    const float K = fmaf(-1.5f * rho, fmaf(c.U, c.U, fmaf(c.V, c.V, c.W * c.W)), d);
    const float sr = sgn * rho * s18;
    c.K1 = K * (1.f / 18.f);
    c.sA1 = sr;
    c.B1 = rho * 0.25f;
    c.K2 = K * (1.f / 36.f);
    c.sA2 = 0.5f * sr;
    c.B2 = rho * 0.125f;
    return c;
}
// K + B e^2 + sA e
__device__ __forceinline__ float nb_val(float K, float sA, float B, float e) { return fmaf(sA, e, fmaf(B * e, e, K)); }

// c.u of the five pairs with c_y = +1: c = (0,1,0), (1,1,0), (-1,1,0), (0,1,1), (0,1,-1)
__device__ __forceinline__ F2 ye2(const NC2 &nc, int k, int j) {
    return k == 0 ? nc.V[j]
                  : (k == 1 ? add2(nc.U[j], nc.V[j])
                            : (k == 2 ? sub2(nc.V[j], nc.U[j])
                                      : (k == 3 ? add2(nc.V[j], nc.W[j]) : sub2(nc.V[j], nc.W[j]))));
}

// shift a lane-distributed row by +1 (g[x] <- g[x-1]) or -1 (g[x] <- g[x+1]);
// the node crossing the lane boundary comes from the neighbouring lane
__device__ __forceinline__ void shift2(F2 (&g)[2], int dir, int lane) {
    if (dir > 0) {
        const float e = __shfl_sync(FULL, g[1].y, (lane + 31) & 31);
        g[1] = make_float2(g[0].y, g[1].x);
        g[0] = make_float2(e, g[0].x);
    } else {
        const float e = __shfl_sync(FULL, g[0].x, (lane + 1) & 31);
        g[0] = make_float2(g[0].y, g[1].x);
        g[1] = make_float2(g[1].y, e);
    }
}

__device__ __forceinline__ void st_slot2(float *slot, const F2 (&o)[2], int lane) {
    *reinterpret_cast<float4 *>(slot + spos(lane, 0)) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
}
__device__ __forceinline__ void ld_slot2(const float *slot, F2 (&o)[2], int lane) {
    const float4 t = *reinterpret_cast<const float4 *>(slot + spos(lane, 0));
    o[0] = make_float2(t.x, t.y);
    o[1] = make_float2(t.z, t.w);
}

// Row-crossing values of one half row, computed once per link pair and sent to
// the receivers above (up, c_y = +1; when UP) and below (down, c_y = -1; when DN),
// four values per receiver x and direction:
//   slot 0: sum of the three c_z = 0 links (d, +-jy), slot 1: their x-momentum,
//   slot 2: the c_z = +1 link, slot 3: the c_z = -1 link.
// With NH = 2 the boundary lanes take the x-shifted diagonal that crosses from the
// other half from the neighbour's values nb1 (c = (1,1,0) at lane 0, (-1,-1,0) at
// lane 31) and nb2 (c = (1,-1,0) at lane 0, (-1,1,0) at lane 31).
// XW (x walls: the cavity's x = 0 and x = nx-1 faces): e0 / eN mark the lane that
// holds node x = 0 / x = nx-1. A value that would cross such a face (wrapped
// periodically) is dropped, and for an own row (own != nullptr) the node takes
// instead its own value of the bounced link (Eq. ACM2.0cccbb2; the moving-wall
// term is zero: the lid is not on an x face): link (1,1,0) arriving at x = 0 is
// replaced by the node's (-1,-1,0) value, and so on.
template <int NH, int MODE, bool XW = false>
__device__ __forceinline__ void send_rows(const NC2 &nc, float *ubase, float *dbase, bool UP, bool DN,
                                          float nb1, float nb2, int lane, bool w0 = false, bool wN = false,
                                          bool e0 = false, bool eN = false, F2 (*own)[4] = nullptr) {
    constexpr int XSLOT = HG<NH>::XSLOT;
    const bool l0 = lane == 0 && HG<NH>::NB, l31 = lane == 31 && HG<NH>::NB;
    if (MODE == MID) {
        F2 u0[2], u1[2], d0[2], d1[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) pair2(nc, j, ye2(nc, 0, j), false, u0[j], d0[j]);  // c = (0,1,0)
        {  // k = 1: c = (1,1,0) [up: receiver x <- x-1]; -c = (-1,-1,0) [down: x <- x+1]
            F2 gp[2], gm[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) pair2(nc, j, ye2(nc, 1, j), true, gp[j], gm[j]);
            if (XW && own) {
                if (w0 && e0) {  // (1,1,0) into x = 0 bounces: its (-1,-1,0) value
                    const float v = gm[0].x;
                    own[0][0].x += v;
                    own[0][1].x += v;
                    own[0][2].x += v;
                }
                if (wN && eN) {  // (-1,-1,0) into x = nx-1 bounces: its (1,1,0) value
                    const float v = gp[1].y;
                    own[1][0].y += v;
                    own[1][1].y -= v;
                    own[1][2].y -= v;
                }
            }
            if (UP) {
                shift2(gp, 1, lane);
                gp[0].x = l0 ? nb1 : gp[0].x;
                if (XW && w0) gp[0].x = e0 ? 0.f : gp[0].x;
            }
            if (DN) {
                shift2(gm, -1, lane);
                gm[1].y = l31 ? nb1 : gm[1].y;
                if (XW && wN) gm[1].y = eN ? 0.f : gm[1].y;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                u0[j] = add2(u0[j], gp[j]);
                u1[j] = gp[j];
                d0[j] = add2(d0[j], gm[j]);
                d1[j] = neg2(gm[j]);
            }
        }
        {  // k = 2: c = (-1,1,0) [up: x <- x+1]; -c = (1,-1,0) [down: x <- x-1]
            F2 gp[2], gm[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) pair2(nc, j, ye2(nc, 2, j), true, gp[j], gm[j]);
            if (XW && own) {
                if (w0 && e0) {  // (1,-1,0) into x = 0 bounces: its (-1,1,0) value
                    const float v = gp[0].x;
                    own[0][0].x += v;
                    own[0][1].x += v;
                    own[0][2].x -= v;
                }
                if (wN && eN) {  // (-1,1,0) into x = nx-1 bounces: its (1,-1,0) value
                    const float v = gm[1].y;
                    own[1][0].y += v;
                    own[1][1].y -= v;
                    own[1][2].y += v;
                }
            }
            if (UP) {
                shift2(gp, -1, lane);
                gp[1].y = l31 ? nb2 : gp[1].y;
                if (XW && wN) gp[1].y = eN ? 0.f : gp[1].y;
            }
            if (DN) {
                shift2(gm, 1, lane);
                gm[0].x = l0 ? nb2 : gm[0].x;
                if (XW && w0) gm[0].x = e0 ? 0.f : gm[0].x;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                u0[j] = add2(u0[j], gp[j]);
                u1[j] = sub2(u1[j], gp[j]);
                d0[j] = add2(d0[j], gm[j]);
                d1[j] = add2(d1[j], gm[j]);
            }
        }
        if (UP) {
            st_slot2(ubase + 0 * XSLOT, u0, lane);
            st_slot2(ubase + 1 * XSLOT, u1, lane);
        }
        if (DN) {
            st_slot2(dbase + 0 * XSLOT, d0, lane);
            st_slot2(dbase + 1 * XSLOT, d1, lane);
        }
    }
    // k = 3: c = (0,1,1), -c = (0,-1,-1); k = 4: c = (0,1,-1), -c = (0,-1,1)
    // slot 2 (c_z = +1): up <- c of k = 3, down <- -c of k = 4
    // slot 3 (c_z = -1): up <- c of k = 4, down <- -c of k = 3
    {
        F2 gp[2], gm[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) pair2(nc, j, ye2(nc, 3, j), true, gp[j], gm[j]);
        if (UP && MODE != LAST) st_slot2(ubase + 2 * XSLOT, gp, lane);
        if (DN && MODE != FIRST) st_slot2(dbase + 3 * XSLOT, gm, lane);
    }
    {
        F2 gp[2], gm[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) pair2(nc, j, ye2(nc, 4, j), true, gp[j], gm[j]);
        if (UP && MODE != FIRST) st_slot2(ubase + 3 * XSLOT, gp, lane);
        if (DN && MODE != LAST) st_slot2(dbase + 2 * XSLOT, gm, lane);
    }
}

// which halves of the in-row pair (c = (1,0,cz), -c) a mode needs
__device__ __forceinline__ constexpr bool need_p(int mode, int cz) {
    return mode == MID || (mode == FIRST ? cz > 0 : cz < 0);
}
__device__ __forceinline__ constexpr bool need_m(int mode, int cz) {
    return mode == MID || (mode == FIRST ? cz < 0 : cz > 0);
}

using Acc = F2[3][2][4];  // [plane behind / current / ahead][node pair][d, jx, jy, jz]

template <int NH, int MODE, bool F, bool XW, typename T>
__device__ __forceinline__ void phase_a(Acc &acc, const T *stg, float *xbuf, const TiledParams &p, int lane,
                                        int row, int half) {
    constexpr int PM = 0, P0 = 1, PP = 2;
    // w0 / wN: the warp holds the x = 0 / x = nx-1 end of its row (warp-uniform, so
    // the other warps skip the face code); e0 / eN: the lane holding that node
    const bool w0 = XW && half == 0, wN = XW && half == NH - 1;
    const bool e0 = w0 && lane == 0, eN = wN && lane == 31;
    constexpr int RL = HG<NH>::RL, XDIR = HG<NH>::XDIR, SRL = HG<NH>::SRL, OWN = HG<NH>::OWN;
    constexpr bool NB = HG<NH>::NB;
    float *up = xbuf + half * HALF, *dn = xbuf + XDIR + half * HALF;
    {
        NC2 nc;
        node_consts2(nc, stg + (row + 1) * SRL + OWN + half * HALF, HGeo<NH>::TRW * SRL, lane, p.s18, p.a, p.am1);
        // the boundary neighbour's constants (NB; unused for NH = 1)
        const int nbx = lane < 16 ? HG<NH>::left(half) : HG<NH>::right(half);
        const float sgn = lane < 16 ? 1.f : -1.f;
        NbC nb{};
        if (NB) nb = nb_consts(stg + (row + 1) * SRL, HGeo<NH>::TRW * SRL, nbx, sgn, p.s18);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            F2 gp, gm;
            pair2(nc, j, nc.W[j], false, gp, gm);  // (0,0,+1) / (0,0,-1)
            if (MODE == MID) {
                acc[P0][j][3] = acc[P0][j][0];                       // jz so far = d so far
                acc[P0][j][0] = fma2(b2(6.f), nc.K1[j], acc[P0][j][0]);  // rest link: w_0 K = K/3
                // post-combine a rho u = u + M u, never rounding the O(1) factor a rho
                acc[P0][j][1] = add2(fma2(nc.M[j], nc.U[j], acc[P0][j][1]), nc.U[j]);
                acc[P0][j][2] = add2(fma2(nc.M[j], nc.V[j], acc[P0][j][2]), nc.V[j]);
                acc[P0][j][3] = add2(fma2(nc.M[j], nc.W[j], acc[P0][j][3]), nc.W[j]);
                if (F) {  // Eq. force: rho(x,t) g = g + d g, the odd part of f^(e)(rho, g)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        acc[P0][j][1 + c] = fma2(nc.D[j], b2(p.g[c]), add2(acc[P0][j][1 + c], b2(p.g[c])));
                }
            }
            if (MODE != LAST) acc[PP][j][0] = gp;  // first value of the plane ahead
            if (MODE != FIRST) {
                acc[PM][j][0] = add2(acc[PM][j][0], gm);
                acc[PM][j][3] = sub2(acc[PM][j][3], gm);
            }
        }
#pragma unroll
        for (int cz = -1; cz <= 1; ++cz) {
            const bool np = need_p(MODE, cz), nm = need_m(MODE, cz);
            if (!np && !nm) continue;
            F2 gp[2], gm[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const F2 e = cz == 0 ? nc.U[j] : (cz > 0 ? add2(nc.U[j], nc.W[j]) : sub2(nc.U[j], nc.W[j]));
                pair2(nc, j, e, cz != 0, gp[j], gm[j]);
            }
            // in-row deposits as packed pairs of receivers: for +c the receivers
            // (0,1 | 2,3) take the values of nodes (-1,0 | 1,2), for -c those of
            // nodes (1,2 | 3,4); nodes -1 and 4 are the neighbouring lanes'
            // NH = 2: lane 0's +c value and lane 31's -c value from the neighbour
            const float nbv = NB ? nb_val(cz ? nb.K2 : nb.K1, cz ? nb.sA2 : nb.sA1, cz ? nb.B2 : nb.B1,
                                          cz == 0 ? nb.U : (cz > 0 ? nb.U + nb.W : nb.U - nb.W))
                                 : 0.f;
            if (XW && MODE == MID) {  // links crossing an x face bounce (see send_rows)
                if (w0 && e0) {  // (1,0,cz) into x = 0: its own (-1,0,-cz) value
                    const float v = gm[0].x;
                    acc[P0][0][0].x += v;
                    acc[P0][0][1].x += v;
                    if (cz) acc[P0][0][3].x += cz * v;
                }
                if (wN && eN) {  // (-1,0,-cz) into x = nx-1: its own (1,0,cz) value
                    const float v = gp[1].y;
                    acc[P0][1][0].y += v;
                    acc[P0][1][1].y -= v;
                    if (cz) acc[P0][1][3].y -= cz * v;
                }
            }
            if (np) {  // c = (1,0,cz): node i feeds node i+1
                const float eP = gp[1].y;
                float rP = __shfl_sync(FULL, eP, (lane + 31) & 31);
                if (NB) rP = lane == 0 ? nbv : rP;
                if (XW && w0) rP = e0 ? 0.f : rP;
                const F2 R[2] = {make_float2(rP, gp[0].x), make_float2(gp[0].y, gp[1].x)};
                F2(&a)[2][4] = acc[pl<PM, P0, PP>(cz)];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    a[j][0] = add2(a[j][0], R[j]);
                    a[j][1] = add2(a[j][1], R[j]);
                    if (cz < 0) a[j][3] = sub2(a[j][3], R[j]);
                }
            }
            if (nm) {  // -c = (-1,0,-cz): node i feeds node i-1
                const float eM = gm[0].x;
                float rM = __shfl_sync(FULL, eM, (lane + 1) & 31);
                if (NB) rM = lane == 31 ? nbv : rM;
                if (XW && wN) rM = eN ? 0.f : rM;
                const F2 L[2] = {make_float2(gm[0].y, gm[1].x), make_float2(gm[1].y, rM)};
                if (cz < 0) {  // -c = (-1,0,1): first x-momentum of the plane ahead
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        acc[PP][j][0] = add2(acc[PP][j][0], L[j]);
                        acc[PP][j][1] = neg2(L[j]);
                    }
                } else {
                    F2(&a)[2][4] = acc[pl<PM, P0, PP>(-cz)];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        a[j][0] = add2(a[j][0], L[j]);
                        a[j][1] = sub2(a[j][1], L[j]);
                        if (cz > 0) a[j][3] = sub2(a[j][3], L[j]);
                    }
                }
            }
        }
        const float nb1 = NB && MODE == MID ? nb_val(nb.K2, nb.sA2, nb.B2, nb.U + nb.V) : 0.f;
        const float nb2 = NB && MODE == MID ? nb_val(nb.K2, -nb.sA2, nb.B2, nb.V - nb.U) : 0.f;
        send_rows<NH, MODE, XW>(nc, up + (row + 1) * RL, dn + (row - 1) * RL, row + 1 < HGeo<NH>::RW, row > 0, nb1, nb2, lane,
                                w0, wN, e0, eN, MODE == MID ? acc[P0] : nullptr);
    }
    // halo rows: y0-1 (staged row 0) feeds row 0, y0+RW (staged RW+1) row RW-1
    if (row == 0 || row == HGeo<NH>::RW - 1) {
        const int sr = row == 0 ? 0 : HGeo<NH>::TRW - 1;
        NC2 hc;
        node_consts2(hc, stg + sr * SRL + OWN + half * HALF, HGeo<NH>::TRW * SRL, lane, p.s18);
        float nb1 = 0.f, nb2 = 0.f;
        if (NB && MODE == MID) {
            const int nbx = lane < 16 ? HG<NH>::left(half) : HG<NH>::right(half);
            const NbC hb = nb_consts(stg + sr * SRL, HGeo<NH>::TRW * SRL, nbx, lane < 16 ? 1.f : -1.f, p.s18);
            nb1 = nb_val(hb.K2, hb.sA2, hb.B2, hb.U + hb.V);
            nb2 = nb_val(hb.K2, -hb.sA2, hb.B2, hb.V - hb.U);
        }
        if (row == 0)
            send_rows<NH, MODE, XW>(hc, up, nullptr, true, false, nb1, nb2, lane, w0, wN, e0, eN);
        else
            send_rows<NH, MODE, XW>(hc, nullptr, dn + (HGeo<NH>::RW - 1) * RL, false, true, nb1, nb2, lane, w0, wN, e0, eN);
    }
}

// SRND: BF16 / FP16 stores rounded stochastically (tile_common.cuh) with the step's key;
// NUPV: omega_p, the density adds sdelta P (P formed before the step by k_nup_sum)
template <int NH, int MODE, bool SRND, bool NUPV, typename T>
__device__ __forceinline__ void phase_b(Acc &acc, const float *xbuf, T *out, const TiledParams &p, int lane,
                                        int row, int half, int col, int x0, int zfin, uint32_t key) {
    constexpr int PM = 0, P0 = 1, PP = 2;
    constexpr int RL = HG<NH>::RL, XDIR = HG<NH>::XDIR, XSLOT = HG<NH>::XSLOT;
    const float *up = xbuf + row * RL + half * HALF, *dn = xbuf + XDIR + row * RL + half * HALF;
    F2 o[2];
    if (MODE == MID) {
        ld_slot2(up, o, lane);  // from below, c_z = 0: d, +jy
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            acc[P0][j][0] = add2(acc[P0][j][0], o[j]);
            acc[P0][j][2] = add2(acc[P0][j][2], o[j]);
        }
        ld_slot2(up + XSLOT, o, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[P0][j][1] = add2(acc[P0][j][1], o[j]);
        ld_slot2(dn, o, lane);  // from above, c_z = 0: d, -jy
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            acc[P0][j][0] = add2(acc[P0][j][0], o[j]);
            acc[P0][j][2] = sub2(acc[P0][j][2], o[j]);
        }
        ld_slot2(dn + XSLOT, o, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[P0][j][1] = add2(acc[P0][j][1], o[j]);
    }
    if (MODE != LAST) {  // c_z = +1 arrivals for the plane ahead (jz implied by d)
        ld_slot2(up + 2 * XSLOT, o, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            acc[PP][j][0] = add2(acc[PP][j][0], o[j]);
            acc[PP][j][2] = o[j];  // first y-momentum of the plane ahead
        }
        ld_slot2(dn + 2 * XSLOT, o, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            acc[PP][j][0] = add2(acc[PP][j][0], o[j]);
            acc[PP][j][2] = sub2(acc[PP][j][2], o[j]);
        }
    }
    if (MODE != FIRST) {  // c_z = -1 arrivals complete the plane behind
        ld_slot2(up + 3 * XSLOT, o, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            acc[PM][j][0] = add2(acc[PM][j][0], o[j]);
            acc[PM][j][2] = add2(acc[PM][j][2], o[j]);
            acc[PM][j][3] = sub2(acc[PM][j][3], o[j]);
        }
        ld_slot2(dn + 3 * XSLOT, o, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            acc[PM][j][0] = add2(acc[PM][j][0], o[j]);
            acc[PM][j][2] = sub2(acc[PM][j][2], o[j]);
            acc[PM][j][3] = sub2(acc[PM][j][3], o[j]);
        }
        // zfin < 0: no plane to store (or the thread's nodes lie beyond ny or nx)
        if (zfin >= 0) {
            const long long rowoff =
                ((long long)zfin * p.ny + col * HGeo<NH>::RW + row) * p.nx + x0 + half * HALF + lane * VXH;
            T *op = out + rowoff;
            if constexpr (NUPV) {  // d+ = sum of the link values + sdelta P (as s_p in place of s)
                const float4 pv = *reinterpret_cast<const float4 *>(p.pfield + rowoff);
                acc[PM][0][0] = fma2(b2(p.sdelta), make_float2(pv.x, pv.y), acc[PM][0][0]);
                acc[PM][1][0] = fma2(b2(p.sdelta), make_float2(pv.z, pv.w), acc[PM][1][0]);
            }
            // u = j / rho, correctly rounded (tile_common.cuh, div_apply2)
            const Div2 r[2] = {div_prep2(add2(b2(1.f), acc[PM][0][0])), div_prep2(add2(b2(1.f), acc[PM][1][0]))};
            if constexpr (SRND && sizeof(T) == 2) {
                // random words of the lane's four nodes: h[0] for d (low) and u (high), h[1] for v and w
                const uint32_t k0 = (uint32_t)rowoff;
                uint32_t h[2][4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    h[0][i] = sr_bits(k0 + i, 0u, key);
                    h[1][i] = sr_bits(k0 + i, 1u, key);
                }
                st4_sr(op, acc[PM][0][0].x, acc[PM][0][0].y, acc[PM][1][0].x, acc[PM][1][0].y, h[0][0], h[0][1],
                       h[0][2], h[0][3]);
#pragma unroll
                for (int c = 1; c < 4; ++c) {
                    const F2 v0 = div_apply2(acc[PM][0][c], r[0]), v1 = div_apply2(acc[PM][1][c], r[1]);
                    const int q = c >> 1, sh = (c & 1) * 16;
                    st4_sr(op + c * p.fstride, v0.x, v0.y, v1.x, v1.y, h[q][0] >> sh, h[q][1] >> sh, h[q][2] >> sh,
                           h[q][3] >> sh);
                }
            } else {
                st4(op, acc[PM][0][0].x, acc[PM][0][0].y, acc[PM][1][0].x, acc[PM][1][0].y);
#pragma unroll
                for (int c = 1; c < 4; ++c) {
                    const F2 v0 = div_apply2(acc[PM][0][c], r[0]), v1 = div_apply2(acc[PM][1][c], r[1]);
                    st4(op + c * p.fstride, v0.x, v0.y, v1.x, v1.y);
                }
            }
        }
    }
}

// NH = 0: the bulk copies of one staged row (field f, row r) of an item, relative to
// the plane's start: from element a, na bytes, then (x wrap) from element b, nb bytes,
// and, for a row shorter than 136 nodes (one segment), the rest of the staged row
// from element b again (the row's start once more). Formed once per item by the
// thread that issues them, kept in shared memory.
struct SegCopy {
    long long a, b;
    int na, nb;
};
constexpr int SEG_COPIES = 4 * (ROWS + 2);  // staged rows per plane (all four fields)

// The staged rows of one plane (four fields) for an item's rows, by 1-D bulk copies
// that complete on `bar`. NH = 1, 2: one thread issues them (the whole rows, wrapped
// in y). NH = 0: 40 staged rows (a segment at an x end of the domain takes its
// wrapped 8 nodes in a second copy), issued by lane 0 of rows 1-6, every sixth row
// each (a bulk copy takes warp-uniform operands, so the lanes of one warp would
// issue theirs one after another, and that warp would hold up the plane barrier),
// from offsets formed once per item (per plane only the plane's offset is added:
// forming them per plane cost ~100 instructions per node); row 1's thread also posts
// the expected bytes (the barrier's transaction count may run below zero until it
// does).
template <int NH, typename T>
__device__ __forceinline__ void issue_plane(const T *in, const TiledParams &p, int col, int z, T *stage,
                                            uint64_t *bar, int warp, SegCopy *dsc = nullptr, int *dcol = nullptr) {
    constexpr int RL = HG<NH, T>::RL, SRL = HG<NH, T>::SRL;
    constexpr uint32_t TX = HG<NH, T>::TX;
    const int zl = z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z);
    const long long plane = (long long)p.nx * p.ny;
    if constexpr (NH == 0) {
        static_assert(4 * HGeo<NH>::TRW == SEG_COPIES, "one descriptor per staged row");
        const int w = warp - 1;  // this thread's rows: k = w, w + 6, ...
        if (warp == 1) mbar_expect_tx(bar, TX);
        if (dcol[w] != col) {  // a new item: form its copies (the row offsets wrapped once here)
            const int seg = col / p.ycols, y0 = (col - seg * p.ycols) * HGeo<NH>::RW;
            const int x0 = seg * HALF, rn = p.nx - x0, last = p.segs - 1;
            for (int k = w; k < SEG_COPIES; k += 6) {
                const int f = k / HGeo<NH>::TRW, r = k - f * HGeo<NH>::TRW;
                const int y = (y0 - 1 + r + p.ny) % p.ny;  // a remainder: rows of a short last column wrap
                const long long rb = f * p.fstride + (long long)y * p.nx;
                SegCopy d;
                if (last == 0) {  // one short segment: the row's last 8 nodes, the row, its start
                    d.a = rb + p.nx - 8, d.na = 8 * (int)sizeof(T), d.b = rb, d.nb = p.nx * (int)sizeof(T);
                } else if (seg == 0) {  // the row's last 8 nodes, then its first 136
                    d.a = rb + p.nx - 8, d.na = 8 * (int)sizeof(T), d.b = rb, d.nb = (HALF + 8) * (int)sizeof(T);
                } else if (seg == last) {  // to the row's end, then the row's start (wrapped)
                    d.a = rb + x0 - 8, d.na = (rn + 8) * (int)sizeof(T), d.b = rb, d.nb = (HALF + 8 - rn) * (int)sizeof(T);
                } else {
                    d.a = rb + x0 - 8, d.na = SRL * (int)sizeof(T), d.b = 0, d.nb = 0;
                }
                dsc[k] = d;
            }
            dcol[w] = col;
        }
        const long long zo = (long long)zl * plane;
        if (p.segs > 1) {
            for (int k = w; k < SEG_COPIES; k += 6) {
                const SegCopy d = dsc[k];
                T *dst = stage + k * SRL;
                bulk_g2s(dst, in + zo + d.a, (uint32_t)d.na, bar);
                if (d.nb) bulk_g2s(dst + d.na / (int)sizeof(T), in + zo + d.b, (uint32_t)d.nb, bar);
            }
        } else {  // one short segment: the row's start a second time fills the staged row
            for (int k = w; k < SEG_COPIES; k += 6) {
                const SegCopy d = dsc[k];
                T *dst = stage + k * SRL;
                const int rest = SRL * (int)sizeof(T) - d.na - d.nb;
                bulk_g2s(dst, in + zo + d.a, (uint32_t)d.na, bar);
                bulk_g2s(dst + d.na / (int)sizeof(T), in + zo + d.b, (uint32_t)d.nb, bar);
                bulk_g2s(dst + (d.na + d.nb) / (int)sizeof(T), in + zo + d.b, (uint32_t)rest, bar);
            }
        }
    } else {
        const int y0 = col * HGeo<NH>::RW;
        mbar_expect_tx(bar, TX);
        const uint32_t rb = (uint32_t)(RL * sizeof(T));
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const T *src = in + f * p.fstride + (long long)zl * plane;
            T *dst = stage + f * HGeo<NH>::TRW * RL;
            if (y0 >= 1 && y0 + HGeo<NH>::RW < p.ny) {
                bulk_g2s(dst, src + (long long)(y0 - 1) * p.nx, HGeo<NH>::TRW * rb, bar);
            } else if (y0 + HGeo<NH>::RW <= p.ny) {
                const int yb = y0 - 1 < 0 ? y0 - 1 + p.ny : y0 - 1;
                const int yt = y0 + HGeo<NH>::RW >= p.ny ? y0 + HGeo<NH>::RW - p.ny : y0 + HGeo<NH>::RW;
                bulk_g2s(dst, src + (long long)yb * p.nx, rb, bar);
                bulk_g2s(dst + RL, src + (long long)y0 * p.nx, HGeo<NH>::RW * rb, bar);
                bulk_g2s(dst + (HGeo<NH>::TRW - 1) * RL, src + (long long)yt * p.nx, rb, bar);
            } else if (p.ny >= HGeo<NH>::TRW) {
                // a short last column (ny % 8 != 0; y0 >= 8): row y0 - 1, its R rows up
                // to ny - 1, then the rows from y = 0 that follow them periodically
                const int R = p.ny - y0;
                bulk_g2s(dst, src + (long long)(y0 - 1) * p.nx, rb, bar);
                bulk_g2s(dst + RL, src + (long long)y0 * p.nx, (uint32_t)R * rb, bar);
                bulk_g2s(dst + (R + 1) * RL, src, (uint32_t)(HGeo<NH>::TRW - 1 - R) * rb, bar);
            } else {  // fewer than 10 rows in all: each staged row by itself, wrapped
                for (int r = 0; r < HGeo<NH>::TRW; ++r)
                    bulk_g2s(dst + r * RL, src + (long long)((y0 - 1 + r + p.ny) % p.ny) * p.nx, rb, bar);
            }
        }
    }
}

// the plane ahead starts from its first deposits (assignments), so it needs no
// clearing; a plane behind that holds values of another run is never stored
__device__ __forceinline__ void rotate(Acc &acc) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[0][j][c] = acc[1][j][c];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[1][j][c] = acc[2][j][c];
    }
}

// V: the variant, 0 = the plain scheme, 1 = with a constant acceleration (Eq. force),
// 2 = with the x faces walled (the cavity's x = 0 and x = nx-1 faces, lid elsewhere),
// 3 = the plain scheme with BF16 / FP16 stores rounded stochastically,
// 4 = the pressure update relaxed with omega_p (periodic, no forcing)
template <int NH, typename T, int V>
__global__ void __launch_bounds__(HG<NH>::NTH, HG<NH>::MINB) k_d3q19_half(const T *__restrict__ in,
                                                                   T *__restrict__ out, TiledParams p) {
    constexpr bool F = V == 1, XW = V == 2, SRND = V == 3, NUPV = V == 4;
    constexpr int XBUF = HG<NH, T>::XBUF, STAGE = HG<NH, T>::STAGE;
    extern __shared__ float4 smem4[];
    float *xs = reinterpret_cast<float *>(smem4);
    T *stg = reinterpret_cast<T *>(xs + 2 * XBUF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg + 2 * STAGE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row = NH == 2 ? warp >> 1 : warp, half = NH == 2 ? (warp & 1) : 0;
    // the thread that issues the copies (NH = 0: lane 0 of rows 1 to 6, see
    // issue_plane): in row 1, which has no halo row to send
    const bool producer = threadIdx.x == (NH == 2 ? 64 : 32);
    const bool issuer = NH == 0 ? (lane == 0 && warp >= 1 && warp <= 6) : producer;
    if ((int)blockIdx.x >= p.nitems) return;  // uniform per CTA
    // programmatic dependent launch: the next step's kernel may be scheduled now; its
    // CTAs take an SM as one of this grid's leaves it and set up their shared memory
    // while the rest run, then wait (griddepcontrol.wait below) for this grid to
    // complete before they touch global memory
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    __shared__ int failed;
    // NH = 0: the current item's copies and, per issuing row, the item they are for
    __shared__ SegCopy seg_dsc[NH == 0 ? SEG_COPIES : 1];
    __shared__ int seg_col[NH == 0 ? 6 : 1];
    if (NH == 0 && threadIdx.x < 6) seg_col[threadIdx.x] = -1;
    if (threadIdx.x == 0) {
        failed = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the grid before this one in the stream (launched with programmatic stream
    // serialization: a no-op otherwise) has completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");

    TaskIter it(blockIdx.x, p.nitems, gridDim.x, p.ycols * p.segs, p.zc, p.nz, p.kcls);
    TaskIter pf = it;
    int issued = 0;
    for (int k = 0; k < 2 && pf.valid(); ++k) {
        if (issuer) issue_plane<NH, T>(in, p, pf.col, pf.pz, stg + k * STAGE, &bars[k], warp, seg_dsc, seg_col);
        ++issued;
        pf.next();
    }

    // the step's random key (the counter advances after the launch, k_sr_tick)
    const uint32_t key = SRND ? sr_key(*p.sr_ctr) : 0u;
    Acc acc;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][j][c] = b2(0.f);

    for (int tc = 0; it.valid(); ++tc) {
        const int s = tc & 1;
        const T *stage = stg + s * STAGE;
        float *xbuf = xs + s * XBUF;
        const bool ok = mbar_wait(&bars[s], (uint32_t)((tc >> 1) & 1));
        const int mode = it.mode();
        if (ok) {
            if (mode == MID) {
                phase_a<NH, MID, F, XW>(acc, stage, xbuf, p, lane, row, half);
            } else if (mode == FIRST) {
                phase_a<NH, FIRST, F, XW>(acc, stage, xbuf, p, lane, row, half);
            } else {
                phase_a<NH, LAST, F, XW>(acc, stage, xbuf, p, lane, row, half);
            }
        }
        if (!ok) failed = 1;  // a wait that gave up, seen by every thread after the barrier
        __syncthreads();
        if (failed) {
            if (producer) {
                atomicExch(p.err, 1);
                for (int t = tc + 1; t < issued; ++t) mbar_wait(&bars[t & 1], (uint32_t)((t >> 1) & 1));
            }
            return;
        }
        if (pf.valid()) {
            if (issuer) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_plane<NH, T>(in, p, pf.col, pf.pz, stg + s * STAGE, &bars[s], warp, seg_dsc, seg_col);
            }
            ++issued;
            pf.next();
        }
        // NH = 0: the item's column of rows and its segment
        const int seg = HG<NH>::SEG ? it.col / p.ycols : 0, ycol = it.col - seg * p.ycols, x0 = seg * HALF;
        if (NUPV && producer && mode == MID) {
            // omega_p: the density terms of this source plane's rows are read when the
            // plane is completed, next iteration; bring them into L2 now
            const float *pr = p.pfield + ((long long)it.pz * p.ny + ycol * HGeo<NH>::RW) * p.nx + x0;
            if (HG<NH>::SEG) {
                const int rn = p.nx - x0 < HALF ? p.nx - x0 : HALF;
                for (int r = 0; r < HGeo<NH>::RW; ++r) prefetch_l2(pr + (long long)r * p.nx, (uint32_t)rn * 4);
            } else {
                prefetch_l2(pr, (uint32_t)(HGeo<NH>::RW * HG<NH>::RL * 4));
            }
        }
        // a short last column's rows beyond ny (they carry the rows that follow
        // periodically, the first feeding the last real row from above like a halo
        // row) are not stored, nor the nodes of a short last segment beyond nx (they
        // carry the row's first nodes, likewise); the check is made here rather than
        // at the store, where it measured 1.2% slower
        const bool live = ycol * HGeo<NH>::RW + row < p.ny && (!HGeo<NH>::SEG || x0 + lane * VXH < p.nx);
        if (mode == MID) {
            phase_b<NH, MID, SRND, NUPV>(acc, xbuf, out, p, lane, row, half, ycol, x0,
                                         it.pz > it.za && live ? it.pz - 1 : -1, key);
            rotate(acc);
        } else if (mode == FIRST) {
            phase_b<NH, FIRST, SRND, NUPV>(acc, xbuf, out, p, lane, row, half, ycol, x0, -1, key);
            rotate(acc);
        } else {
            phase_b<NH, LAST, SRND, NUPV>(acc, xbuf, out, p, lane, row, half, ycol, x0, live ? it.zb - 1 : -1, key);
        }
        it.next();
    }
}

// per device: opt in to the shared-memory size; persistent grid = CTAs per SM x
// SMs (-1 when a CTA does not fit)
template <int NH, typename T, int V>
cudaError_t prepare(int *ctas) {
    static DevSlots slots;
    const int n = per_device(slots, [] {
        if (cudaFuncSetAttribute(k_d3q19_half<NH, T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)HG<NH, T>::BYTES) != cudaSuccess)
            return -1;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_d3q19_half<NH, T, V>, HG<NH, T>::NTH,
                                                          HG<NH, T>::BYTES) != cudaSuccess || nb < 1)
            return -1;
        return nb * device_sms();
    });
    if (ctas) *ctas = n;
    return n > 0 ? cudaSuccess : cudaErrorNotSupported;
}

}  // namespace

template <int NH, int V>
static cudaError_t prepare_storage(int storage) {
    if constexpr (NH == 0 && V == 2) return cudaErrorNotSupported;  // x walls: rows of 128 / 256 only
    switch (storage) {
        case STORE_F32:
            if constexpr (V == 3) return cudaErrorNotSupported;  // FP32 stores round to nearest
            else return prepare<NH, float, V>(nullptr);
        case STORE_BF16: return prepare<NH, __nv_bfloat16, V>(nullptr);
        case STORE_F16: return prepare<NH, __half, V>(nullptr);
    }
    return cudaErrorInvalidValue;
}

// row geometry (the NH of HG) for a row of nx nodes: 2 (256), 1 (128), 0 (128 S, S >= 3)
static int half_geometry(int nx) { return nx == 256 ? 2 : (nx == 128 ? 1 : 0); }

// rows the segment form takes: at least 72 nodes (a row of one segment is staged as
// its last 8 nodes, itself and its first 136 - nx again: the last must fit in it), a
// last segment of at least 8 nodes (the one before it stages 8 past its end), and
// 16-byte row starts and copy sizes (nx a multiple of 16 bytes' worth)
static bool segments_fit(int nx, int storage) {
    const int q = storage == STORE_F32 ? 4 : 8;
    return nx >= 72 && nx % q == 0 && (nx % HALF == 0 || nx % HALF >= 8);
}

bool half_xwalls(const StepParams &p) {
    return p.walled[0] && p.lid_axis != 0 && half_geometry(p.nx) != 0;
}

// the kernel variant a step needs (-1: none serves it)
static int half_variant(const StepParams &p) {
    const bool walls = p.walled[0] || p.walled[1] || p.walled[2];
    if (p.sr_ctr)  // stochastic rounding: the plain periodic scheme only
        return (walls || p.has_force || p.sdelta != 0.f) ? -1 : 3;
    if (p.sdelta != 0.f)  // omega_p: periodic, no forcing, with its scratch field
        return (walls || p.has_force || !p.nup_p || !nup_sum_supported(p)) ? -1 : 4;
    const bool xw = half_xwalls(p);
    if (p.has_force && xw) return -1;
    return xw ? 2 : (p.has_force ? 1 : 0);
}

bool half_supported(int Q, int storage, const StepParams &p) {
    if (Q != 19) return false;
    // walled domains (cavity, channel): the kernel wraps every axis and the wall pass
    // after it recomputes every boundary node, the only nodes with a source outside
    if (storage != STORE_F32 && storage != STORE_BF16 && storage != STORE_F16) return false;
    // the plain scheme, with or without a constant acceleration (Eq. force)
    if (p.gfield || p.scalar || p.bulk) return false;
    if (p.ny < 1 || p.nz < 1) return false;
    if (half_geometry(p.nx) == 0 && !segments_fit(p.nx, storage)) return false;
    if (p.fstride % 8 != 0 || !p.err) return false;  // 16-byte field starts for 2-byte storage
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const int v = half_variant(p);
    if (v < 0) return false;
    cudaError_t e;
    const int g = half_geometry(p.nx);
    if (g == 2)
        e = v == 0   ? prepare_storage<2, 0>(storage)
            : v == 1 ? prepare_storage<2, 1>(storage)
            : v == 2 ? prepare_storage<2, 2>(storage)
            : v == 3 ? prepare_storage<2, 3>(storage)
                     : prepare_storage<2, 4>(storage);
    else if (g == 1)
        e = v == 0   ? prepare_storage<1, 0>(storage)
            : v == 1 ? prepare_storage<1, 1>(storage)
            : v == 2 ? prepare_storage<1, 2>(storage)
            : v == 3 ? prepare_storage<1, 3>(storage)
                     : prepare_storage<1, 4>(storage);
    else
        e = v == 0   ? prepare_storage<0, 0>(storage)
            : v == 1 ? prepare_storage<0, 1>(storage)
            : v == 3 ? prepare_storage<0, 3>(storage)
                     : prepare_storage<0, 4>(storage);
    return e == cudaSuccess;
}

template <int NH, typename T, int V>
static cudaError_t launch_nh(const void *in, void *out, const StepParams &sp, cudaStream_t st) {
    int ctas = 0;
    cudaError_t e = prepare<NH, T, V>(&ctas);
    if (e != cudaSuccess) return e;
    TiledParams p;
    p.nx = sp.nx;
    p.ny = sp.ny;
    p.nz = sp.nz;
    p.ycols = (sp.ny + HGeo<NH>::RW - 1) / HGeo<NH>::RW;
    p.segs = NH == 0 ? (sp.nx + HALF - 1) / HALF : 1;
    const Schedule sc = plan_schedule(p.ycols * p.segs, sp.nz, ctas);
    p.zc = sc.zc;
    p.nitems = sc.nitems;
    p.kcls = sc.kcls;
    p.fstride = sp.fstride;
    const double nu = (double)sp.s / 18.0;
    p.s18 = (float)nu;
    p.a = sp.a;
    p.am1 = sp.am1;
    p.err = sp.err;
    for (int c = 0; c < 3; ++c) p.g[c] = V == 1 ? sp.force[c] : 0.f;
    p.sr_ctr = V == 3 ? sp.sr_ctr : nullptr;
    p.pfield = V == 4 ? sp.nup_p : nullptr;
    p.sdelta = V == 4 ? sp.sdelta : 0.f;
    // launched with programmatic stream serialization: its CTAs may start before the
    // previous kernel in the stream has finished and wait for it in the kernel (+0.5%
    // on 256^3, +2% on 128^3, where the gap between steps weighs more)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sc.grid);
    cfg.blockDim = dim3(HG<NH, T>::NTH);
    cfg.dynamicSmemBytes = HG<NH, T>::BYTES;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_d3q19_half<NH, T, V>, (const T *)in, (T *)out, p);
}

template <int V, typename T>
static cudaError_t launch_geometry(const void *in, void *out, const StepParams &sp, cudaStream_t st) {
    const int g = half_geometry(sp.nx);
    if (g == 2) return launch_nh<2, T, V>(in, out, sp, st);
    if (g == 1) return launch_nh<1, T, V>(in, out, sp, st);
    if constexpr (V == 2) return cudaErrorNotSupported;
    else return launch_nh<0, T, V>(in, out, sp, st);
}

template <int V>
static cudaError_t launch_variant(int storage, const void *in, void *out, const StepParams &sp, cudaStream_t st) {
    switch (storage) {
        case STORE_F32:
            if constexpr (V == 3) return cudaErrorNotSupported;
            else return launch_geometry<V, float>(in, out, sp, st);
        case STORE_BF16: return launch_geometry<V, __nv_bfloat16>(in, out, sp, st);
        case STORE_F16: return launch_geometry<V, __half>(in, out, sp, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_half(int Q, int storage, const void *in, void *out, const StepParams &sp,
                             cudaStream_t st) {
    if (!half_supported(Q, storage, sp)) return cudaErrorNotSupported;
    const int v = half_variant(sp);
    return v == 0   ? launch_variant<0>(storage, in, out, sp, st)
           : v == 1 ? launch_variant<1>(storage, in, out, sp, st)
           : v == 2 ? launch_variant<2>(storage, in, out, sp, st)
           : v == 3 ? launch_variant<3>(storage, in, out, sp, st)
                    : launch_variant<4>(storage, in, out, sp, st);
}

// advance the stochastic-rounding step counter (after each step's stores)
static __global__ void k_sr_tick(unsigned *ctr) {
    if (threadIdx.x == 0) *ctr += 1u;
}
cudaError_t launch_sr_tick(unsigned *ctr, cudaStream_t st) {
    k_sr_tick<<<1, 32, 0, st>>>(ctr);
    return cudaGetLastError();
}

}  // namespace lwacm
