// Row-tiled update of the passive scalar of Eq. ACM2.0t (thermal LW-ACM,
// Appendix "Asymptotic analysis for energy equation") for periodic D3Q19 domains
// with nx = 128 NH and ny a multiple of 8, FP32 storage. It runs after the flow
// step and reads the same state at t:
//
//     T+(x) = a_t T(x) + sum_i h_i(x - c_i),
//     h_i(y) = w_i [(1 - a_t)(T + 9/2 e^2 - 3/2 |u|^2) + 3 T e](y),   e = c_i . u(y)
//
// (the populations g_i = g^(e)_i(x - c_i) + a_t [g^(e,e)_i(x) - g^(e,e)_i(x - c_i)]
// summed over i; a_t = 1 - 6 alpha; the even part of g^(e) sums to T at a node).
//
// Same organisation as the half-row flow kernel (kernels_half.cu): persistent CTAs
// over (8-row column, run of planes) items with the same schedule, the rows of (T, u, v, w) a plane needs staged
// by 1-D bulk copies (two stages), each source node computing its link values once
// per link pair (c, -c) and depositing them: along x inside a lane or by warp
// shuffle (the two halves of a 256-node row recompute the few values they take from
// each other's boundary node), along y through three exchange slots per receiver
// and direction in shared memory (the c_z = 0 links summed, the c_z = +1 link, the
// c_z = -1 link), along z through three rotating accumulator planes. The scalar has
// one accumulator per node where the flow has four.
#include <stdint.h>

#include "dev_cache.h"
#include "launch.h"
#include "lwacm_core.cuh"
#include "tile_common.cuh"

namespace lwacm {
namespace {

using namespace tile;

constexpr int SHALF = 128;  // nodes per warp row segment (four per lane)
constexpr int SSLOT = 3;    // exchange values per receiver and direction

template <int NH>
struct SG {
    static constexpr int NTH = ROWS * NH * 32;
    static constexpr int RL = SHALF * NH;  // nx
    static constexpr int XSLOT = ROWS * RL;
    static constexpr int XDIR = SSLOT * XSLOT;
    static constexpr int XBUF = 2 * XDIR;
    static constexpr int STAGE = 4 * TROWS * RL;  // T, u, v, w
    static constexpr size_t BYTES = 2 * (size_t)XBUF * 4 + 2 * (size_t)STAGE * 4 + 64;
    static constexpr uint32_t TX = STAGE * 4;
};

struct ScalarParams {
    int nx, ny, nz, ycols, zc, nitems, kcls;  // the schedule (TaskIter, tile_common.cuh)
    long long fstride;
    float at, b1, b2;  // a_t; (1 - a_t) 9/2 w for w = 1/18 and 1/36
    float kt;          // 1 - a_t
    int *err;
};

// The four nodes of a lane are held as two pairs, (0,1) and (2,3), in FP32x2
// registers: the same operation on two nodes issues as one packed instruction (same
// rounding). Unlike the flow kernel, this one has FMA-pipe capacity to spare, so the
// link-pair values are packed too.
using F2 = float2;
__device__ __forceinline__ F2 b2(float v) { return make_float2(v, v); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }

// per node pair: the link-value coefficients of each weight class,
// h = K + e (B e +- O): K = w (1 - a_t)(T - 3/2 |u|^2), O = 3 w T (nO = -O), B uniform
struct SC {
    F2 U[2], V[2], W[2], K1[2], O1[2], nO1[2], K2[2], O2[2], nO2[2], KR[2];  // KR: the rest link + a_t T
};

__device__ __forceinline__ void s_consts(SC &c, const float *row, int rstride, int lane, const ScalarParams &p) {
    const float4 t4 = ld4(row + lane * 4), u4 = ld4(row + rstride + lane * 4);
    const float4 v4 = ld4(row + 2 * rstride + lane * 4), w4 = ld4(row + 3 * rstride + lane * 4);
    const F2 tt[2] = {make_float2(t4.x, t4.y), make_float2(t4.z, t4.w)};
    c.U[0] = make_float2(u4.x, u4.y);
    c.U[1] = make_float2(u4.z, u4.w);
    c.V[0] = make_float2(v4.x, v4.y);
    c.V[1] = make_float2(v4.z, v4.w);
    c.W[0] = make_float2(w4.x, w4.y);
    c.W[1] = make_float2(w4.z, w4.w);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const F2 q = fma2(c.U[j], c.U[j], fma2(c.V[j], c.V[j], mul2(c.W[j], c.W[j])));
        const F2 K = mul2(b2(p.kt), fma2(b2(-1.5f), q, tt[j]));  // (1 - a_t)(T - 3/2 q)
        c.K1[j] = mul2(K, b2(1.f / 18.f));
        c.K2[j] = mul2(K, b2(1.f / 36.f));
        c.O1[j] = mul2(tt[j], b2(1.f / 6.f));     // 3 T / 18
        c.nO1[j] = mul2(tt[j], b2(-1.f / 6.f));
        c.O2[j] = mul2(tt[j], b2(1.f / 12.f));    // 3 T / 36
        c.nO2[j] = mul2(tt[j], b2(-1.f / 12.f));
        c.KR[j] = fma2(b2(p.at), tt[j], mul2(K, b2(1.f / 3.f)));
    }
}

// the pair (c, -c) at node pair j: K + B e^2 +- O e
__device__ __forceinline__ void s_pair(const SC &c, int j, F2 e, bool diag, float b1, float b2v, F2 &hp, F2 &hm) {
    const F2 cm = fma2(mul2(b2(diag ? b2v : b1), e), e, diag ? c.K2[j] : c.K1[j]);
    hp = fma2(diag ? c.O2[j] : c.O1[j], e, cm);
    hm = fma2(diag ? c.nO2[j] : c.nO1[j], e, cm);
}

// the boundary neighbour of a half row (NH = 2): lanes 0-15 take node x0 - 1,
// lanes 16-31 node x0 + 128; sO = +O for lanes 0-15 and -O for lanes 16-31
struct SN {
    float U, V, W, K1, sO1, K2, sO2;
};
__device__ __forceinline__ SN s_nb(const float *row, int rstride, int nbx, float sgn, const ScalarParams &p) {
    SN c;
    const float t = row[nbx];
    c.U = row[rstride + nbx];
    c.V = row[2 * rstride + nbx];
    c.W = row[3 * rstride + nbx];
    const float K = p.kt * fmaf(-1.5f, fmaf(c.U, c.U, fmaf(c.V, c.V, c.W * c.W)), t);
    c.K1 = K * (1.f / 18.f);
    c.K2 = K * (1.f / 36.f);
    c.sO1 = sgn * t * (1.f / 6.f);
    c.sO2 = sgn * t * (1.f / 12.f);
    return c;
}
__device__ __forceinline__ float s_nbv(float K, float sO, float B, float e) { return fmaf(sO, e, fmaf(B * e, e, K)); }

// c.u of the five pairs with c_y = +1: (0,1,0), (1,1,0), (-1,1,0), (0,1,1), (0,1,-1)
__device__ __forceinline__ F2 s_ye(const SC &c, int k, int j) {
    const F2 u = c.U[j], v = c.V[j], w = c.W[j];
    return k == 0 ? v
                  : (k == 1 ? add2(u, v)
                            : (k == 2 ? fma2(u, b2(-1.f), v) : (k == 3 ? add2(v, w) : fma2(w, b2(-1.f), v))));
}

// shift four lane-held values by +1 (g[x] <- g[x-1]) or -1 (g[x] <- g[x+1])
__device__ __forceinline__ void s_shift(F2 (&g)[2], int dir, int lane) {
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
__device__ __forceinline__ void s_st(float *slot, const F2 (&o)[2], int lane) {
    *reinterpret_cast<float4 *>(slot + spos(lane, 0)) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
}
__device__ __forceinline__ void s_ld(const float *slot, F2 (&o)[2], int lane) {
    const float4 t = *reinterpret_cast<const float4 *>(slot + spos(lane, 0));
    o[0] = make_float2(t.x, t.y);
    o[1] = make_float2(t.z, t.w);
}

// The row-crossing values of one half row, sent up (c_y = +1, when UP) and down
// (when DN): slot 0 the sum of the three c_z = 0 links, slot 1 the c_z = +1 link
// (plane ahead), slot 2 the c_z = -1 link (plane behind). NH = 2: the boundary
// lanes take the x-shifted diagonal from the other half's node (nb1: c = (1,1,0)
// at lane 0, (-1,-1,0) at lane 31; nb2: c = (1,-1,0) at lane 0, (-1,1,0) at lane 31).
template <int NH, int MODE>
__device__ __forceinline__ void s_send(const SC &c, const ScalarParams &p, float *ub, float *db, bool UP, bool DN,
                                       float nb1, float nb2, int lane) {
    constexpr int XSLOT = SG<NH>::XSLOT;
    const bool l0 = lane == 0 && NH == 2, l31 = lane == 31 && NH == 2;
    if (MODE == MID) {
        F2 u0[2], d0[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) s_pair(c, j, s_ye(c, 0, j), false, p.b1, p.b2, u0[j], d0[j]);
#pragma unroll
        for (int k = 1; k <= 2; ++k) {  // k = 1: (1,1,0) up x <- x-1, (-1,-1,0) down x <- x+1; k = 2 mirrored
            F2 hp[2], hm[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) s_pair(c, j, s_ye(c, k, j), true, p.b1, p.b2, hp[j], hm[j]);
            if (UP) {
                s_shift(hp, k == 1 ? 1 : -1, lane);
                if (k == 1) hp[0].x = l0 ? nb1 : hp[0].x;
                else hp[1].y = l31 ? nb2 : hp[1].y;
            }
            if (DN) {
                s_shift(hm, k == 1 ? -1 : 1, lane);
                if (k == 1) hm[1].y = l31 ? nb1 : hm[1].y;
                else hm[0].x = l0 ? nb2 : hm[0].x;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                u0[j] = add2(u0[j], hp[j]);
                d0[j] = add2(d0[j], hm[j]);
            }
        }
        if (UP) s_st(ub, u0, lane);
        if (DN) s_st(db, d0, lane);
    }
    {  // k = 3: c = (0,1,1) up -> ahead, -c = (0,-1,-1) down -> behind
        F2 hp[2], hm[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) s_pair(c, j, s_ye(c, 3, j), true, p.b1, p.b2, hp[j], hm[j]);
        if (UP && MODE != LAST) s_st(ub + XSLOT, hp, lane);
        if (DN && MODE != FIRST) s_st(db + 2 * XSLOT, hm, lane);
    }
    {  // k = 4: c = (0,1,-1) up -> behind, -c = (0,-1,1) down -> ahead
        F2 hp[2], hm[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) s_pair(c, j, s_ye(c, 4, j), true, p.b1, p.b2, hp[j], hm[j]);
        if (UP && MODE != FIRST) s_st(ub + 2 * XSLOT, hp, lane);
        if (DN && MODE != LAST) s_st(db + XSLOT, hm, lane);
    }
}

using SAcc = F2[3][2];  // [plane behind / current / ahead][node pair]

template <int NH, int MODE>
__device__ __forceinline__ void s_phase_a(SAcc &acc, const float *stg, float *xbuf, const ScalarParams &p,
                                          int lane, int row, int half) {
    constexpr int PM = 0, P0 = 1, PP = 2;
    constexpr int RL = SG<NH>::RL, XDIR = SG<NH>::XDIR;
    float *up = xbuf + half * SHALF, *dn = xbuf + XDIR + half * SHALF;
    const int nbx = lane < 16 ? (half * SHALF + RL - 1) % RL : (half * SHALF + SHALF) % RL;
    const float sgn = lane < 16 ? 1.f : -1.f;
    {
        SC c;
        s_consts(c, stg + (row + 1) * RL + half * SHALF, TROWS * RL, lane, p);
        SN nb{};
        if (NH == 2) nb = s_nb(stg + (row + 1) * RL, TROWS * RL, nbx, sgn, p);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            F2 hp, hm;
            s_pair(c, j, c.W[j], false, p.b1, p.b2, hp, hm);  // (0,0,+1) / (0,0,-1)
            if (MODE == MID) acc[P0][j] = add2(acc[P0][j], c.KR[j]);  // rest link and a_t T(x)
            if (MODE != LAST) acc[PP][j] = hp;                          // first value of the plane ahead
            if (MODE != FIRST) acc[PM][j] = add2(acc[PM][j], hm);
        }
#pragma unroll
        for (int cz = -1; cz <= 1; ++cz) {
            const bool np = MODE == MID || (MODE == FIRST ? cz > 0 : cz < 0);
            const bool nm = MODE == MID || (MODE == FIRST ? cz < 0 : cz > 0);
            if (!np && !nm) continue;
            F2 hp[2], hm[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const F2 e = cz == 0 ? c.U[j] : (cz > 0 ? add2(c.U[j], c.W[j]) : fma2(c.W[j], b2(-1.f), c.U[j]));
                s_pair(c, j, e, cz != 0, p.b1, p.b2, hp[j], hm[j]);
            }
            const float nbv = NH == 2 ? s_nbv(cz ? nb.K2 : nb.K1, cz ? nb.sO2 : nb.sO1, cz ? p.b2 : p.b1,
                                              cz == 0 ? nb.U : (cz > 0 ? nb.U + nb.W : nb.U - nb.W))
                                      : 0.f;
            if (np) {  // c = (1,0,cz): node n feeds node n+1 in plane +cz
                float r = __shfl_sync(FULL, hp[1].y, (lane + 31) & 31);
                if (NH == 2) r = lane == 0 ? nbv : r;
                const F2 R[2] = {make_float2(r, hp[0].x), make_float2(hp[0].y, hp[1].x)};
                F2(&a)[2] = acc[pl<PM, P0, PP>(cz)];
                a[0] = add2(a[0], R[0]);
                a[1] = add2(a[1], R[1]);
            }
            if (nm) {  // -c = (-1,0,-cz): node n feeds node n-1 in plane -cz
                float r = __shfl_sync(FULL, hm[0].x, (lane + 1) & 31);
                if (NH == 2) r = lane == 31 ? nbv : r;
                const F2 Lv[2] = {make_float2(hm[0].y, hm[1].x), make_float2(hm[1].y, r)};
                F2(&a)[2] = acc[pl<PM, P0, PP>(-cz)];
                a[0] = add2(a[0], Lv[0]);
                a[1] = add2(a[1], Lv[1]);
            }
        }
        const float nb1 = NH == 2 && MODE == MID ? s_nbv(nb.K2, nb.sO2, p.b2, nb.U + nb.V) : 0.f;
        const float nb2 = NH == 2 && MODE == MID ? s_nbv(nb.K2, -nb.sO2, p.b2, nb.V - nb.U) : 0.f;
        s_send<NH, MODE>(c, p, up + (row + 1) * RL, dn + (row - 1) * RL, row + 1 < ROWS, row > 0, nb1, nb2, lane);
    }
    if (row == 0 || row == ROWS - 1) {  // halo rows: y0-1 (staged row 0) feeds row 0, y0+8 (staged 9) row 7
        const int sr = row == 0 ? 0 : TROWS - 1;
        SC h;
        s_consts(h, stg + sr * RL + half * SHALF, TROWS * RL, lane, p);
        float nb1 = 0.f, nb2 = 0.f;
        if (NH == 2 && MODE == MID) {
            const SN hb = s_nb(stg + sr * RL, TROWS * RL, nbx, sgn, p);
            nb1 = s_nbv(hb.K2, hb.sO2, p.b2, hb.U + hb.V);
            nb2 = s_nbv(hb.K2, -hb.sO2, p.b2, hb.V - hb.U);
        }
        if (row == 0)
            s_send<NH, MODE>(h, p, up, nullptr, true, false, nb1, nb2, lane);
        else
            s_send<NH, MODE>(h, p, nullptr, dn + (ROWS - 1) * RL, false, true, nb1, nb2, lane);
    }
}

template <int NH, int MODE>
__device__ __forceinline__ void s_phase_b(SAcc &acc, const float *xbuf, float *tout, const ScalarParams &p,
                                          int lane, int row, int half, int col, int zfin) {
    constexpr int PM = 0, P0 = 1, PP = 2;
    constexpr int RL = SG<NH>::RL, XDIR = SG<NH>::XDIR, XSLOT = SG<NH>::XSLOT;
    const float *up = xbuf + row * RL + half * SHALF, *dn = xbuf + XDIR + row * RL + half * SHALF;
    F2 o[2], q[2];
    if (MODE == MID) {
        s_ld(up, o, lane);
        s_ld(dn, q, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[P0][j] = add2(acc[P0][j], add2(o[j], q[j]));
    }
    if (MODE != LAST) {
        s_ld(up + XSLOT, o, lane);
        s_ld(dn + XSLOT, q, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[PP][j] = add2(acc[PP][j], add2(o[j], q[j]));
    }
    if (MODE != FIRST) {
        s_ld(up + 2 * XSLOT, o, lane);
        s_ld(dn + 2 * XSLOT, q, lane);
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[PM][j] = add2(acc[PM][j], add2(o[j], q[j]));
        if (zfin >= 0) {
            const long long off = ((long long)zfin * p.ny + col * ROWS + row) * p.nx + half * SHALF + lane * 4;
            *reinterpret_cast<float4 *>(tout + off) =
                make_float4(acc[PM][0].x, acc[PM][0].y, acc[PM][1].x, acc[PM][1].y);
        }
    }
}

// (T, u, v, w) of source plane z, rows y0-1 .. y0+8 (periodic)
template <int NH>
__device__ __forceinline__ void s_issue(const float *in, const ScalarParams &p, int col, int z, float *stage,
                                        uint64_t *bar) {
    constexpr int RL = SG<NH>::RL;
    const int zl = z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z);
    const int y0 = col * ROWS;
    const long long plane = (long long)p.nx * p.ny;
    mbar_expect_tx(bar, SG<NH>::TX);
    constexpr uint32_t rb = RL * 4;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int field = f == 0 ? 4 : f;  // T is stored after d, u, v, w
        const float *src = in + field * p.fstride + (long long)zl * plane;
        float *dst = stage + f * TROWS * RL;
        if (y0 >= 1 && y0 + ROWS < p.ny) {
            bulk_g2s(dst, src + (long long)(y0 - 1) * p.nx, TROWS * rb, bar);
        } else {
            const int yb = y0 - 1 < 0 ? y0 - 1 + p.ny : y0 - 1;
            const int yt = y0 + ROWS >= p.ny ? y0 + ROWS - p.ny : y0 + ROWS;
            bulk_g2s(dst, src + (long long)yb * p.nx, rb, bar);
            bulk_g2s(dst + RL, src + (long long)y0 * p.nx, ROWS * rb, bar);
            bulk_g2s(dst + (TROWS - 1) * RL, src + (long long)yt * p.nx, rb, bar);
        }
    }
}

template <int NH>
__global__ void __launch_bounds__(SG<NH>::NTH, 2 / NH) k_scalar_rows(const float *__restrict__ in,
                                                                    float *__restrict__ out, ScalarParams p) {
    constexpr int XBUF = SG<NH>::XBUF, STAGE = SG<NH>::STAGE;
    extern __shared__ float4 smem4[];
    float *xs = reinterpret_cast<float *>(smem4);
    float *stg = xs + 2 * XBUF;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg + 2 * STAGE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row = NH == 2 ? warp >> 1 : warp, half = NH == 2 ? (warp & 1) : 0;
    const bool producer = threadIdx.x == (NH == 2 ? 64 : 32);  // a thread of row 1 (no halo row)
    if ((int)blockIdx.x >= p.nitems) return;
    float *tout = out + 4 * p.fstride;

    __shared__ int failed;
    if (threadIdx.x == 0) {
        failed = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    TaskIter it(blockIdx.x, p.nitems, gridDim.x, p.ycols, p.zc, p.nz, p.kcls);
    TaskIter pf = it;
    int issued = 0;
    for (int k = 0; k < 2 && pf.valid(); ++k) {
        if (producer) s_issue<NH>(in, p, pf.col, pf.pz, stg + k * STAGE, &bars[k]);
        ++issued;
        pf.next();
    }
    SAcc acc;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[a][j] = b2(0.f);

    for (int tc = 0; it.valid(); ++tc) {
        const int s = tc & 1;
        const float *stage = stg + s * STAGE;
        float *xbuf = xs + s * XBUF;
        const bool ok = mbar_wait(&bars[s], (uint32_t)((tc >> 1) & 1));
        const int mode = it.mode();
        if (ok) {
            if (mode == MID)
                s_phase_a<NH, MID>(acc, stage, xbuf, p, lane, row, half);
            else if (mode == FIRST)
                s_phase_a<NH, FIRST>(acc, stage, xbuf, p, lane, row, half);
            else
                s_phase_a<NH, LAST>(acc, stage, xbuf, p, lane, row, half);
        }
        if (!ok) failed = 1;
        __syncthreads();
        if (failed) {
            if (producer) {
                atomicExch(p.err, 1);
                for (int t = tc + 1; t < issued; ++t) mbar_wait(&bars[t & 1], (uint32_t)((t >> 1) & 1));
            }
            return;
        }
        if (pf.valid()) {
            if (producer) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                s_issue<NH>(in, p, pf.col, pf.pz, stg + s * STAGE, &bars[s]);
            }
            ++issued;
            pf.next();
        }
        if (mode == MID) {
            s_phase_b<NH, MID>(acc, xbuf, tout, p, lane, row, half, it.col, it.pz > it.za ? it.pz - 1 : -1);
        } else if (mode == FIRST) {
            s_phase_b<NH, FIRST>(acc, xbuf, tout, p, lane, row, half, it.col, -1);
        } else {
            s_phase_b<NH, LAST>(acc, xbuf, tout, p, lane, row, half, it.col, it.zb - 1);
        }
        if (mode != LAST) {  // rotate: the plane ahead starts from assignments
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                acc[0][j] = acc[1][j];
                acc[1][j] = acc[2][j];
            }
        }
        it.next();
    }
}

template <int NH>
int scalar_ctas() {
    static DevSlots slots;
    return per_device(slots, [] {
        if (cudaFuncSetAttribute(k_scalar_rows<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SG<NH>::BYTES) != cudaSuccess)
            return -1;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scalar_rows<NH>, SG<NH>::NTH, SG<NH>::BYTES) !=
                cudaSuccess ||
            nb < 1)
            return -1;
        return nb * device_sms();
    });
}

}  // namespace

bool scalar_rows_supported(int Q, int storage, const StepParams &p) {
    if (Q != 19 || storage != STORE_F32 || !p.scalar || p.bc != BC_PERIODIC) return false;
    if ((p.nx != 128 && p.nx != 256) || p.ny % ROWS != 0 || p.ny < ROWS || p.nz < 1) return false;
    if (p.fstride % 4 != 0 || !p.err) return false;
    return (p.nx == 256 ? scalar_ctas<2>() : scalar_ctas<1>()) > 0;
}

template <int NH>
static cudaError_t launch_scalar_nh(const void *in, void *out, const StepParams &sp, cudaStream_t st) {
    const int ctas = scalar_ctas<NH>();
    if (ctas < 1) return cudaErrorNotSupported;
    ScalarParams p;
    p.nx = sp.nx;
    p.ny = sp.ny;
    p.nz = sp.nz;
    p.ycols = sp.ny / ROWS;
    const Schedule sc = plan_schedule(p.ycols, sp.nz, ctas);
    p.zc = sc.zc;
    p.nitems = sc.nitems;
    p.kcls = sc.kcls;
    p.fstride = sp.fstride;
    p.at = sp.at;
    p.kt = 1.f - sp.at;
    p.b1 = p.kt * (4.5f / 18.f);
    p.b2 = p.kt * (4.5f / 36.f);
    p.err = sp.err;
    k_scalar_rows<NH><<<(unsigned)sc.grid, SG<NH>::NTH, SG<NH>::BYTES, st>>>((const float *)in, (float *)out, p);
    return cudaGetLastError();
}

cudaError_t launch_scalar_rows(const void *in, void *out, const StepParams &sp, cudaStream_t st) {
    return sp.nx == 256 ? launch_scalar_nh<2>(in, out, sp, st) : launch_scalar_nh<1>(in, out, sp, st);
}

}  // namespace lwacm
