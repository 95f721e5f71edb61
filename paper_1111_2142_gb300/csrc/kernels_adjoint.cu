// Adjoint (reverse-mode derivative) of one LW-ACM step in the moment form, with
// optional forcing and link-wise walls.
//
// Forward step (see lwacm_core.cuh), per receiver x and link i with source
// y = x - c_i, e = c_i . u(y), q = |u(y)|^2, rho = 1 + d:
//     g_i(y)  = w_i [d(y) + rho(y) (s e + 9/2 e^2 - 3/2 q)],      s = 18 nu
//     d+(x)   = sum_i g_i(x - c_i)
//     j+(x)   = a rho(x) u(x) + sum_i c_i g_i(x - c_i) + rho(x) G, a = 1 - 6 nu
//     u+(x)   = j+(x) / (1 + d+(x))
// Given lambda+ = (dL/dd+, dL/du+) at t+1:
//     Jbar(x) = lambda_u+(x) / rho+(x)                              (dL/dj+)
//     Dbar(x) = lambda_d+(x) - lambda_u+(x) . u+(x) / rho+(x)        (dL/dd+, total)
//     gbar_i(y) = Dbar(y + c_i) + c_i . Jbar(y + c_i)                (gathered downwind)
//     lambda_d(y) = sum_i gbar_i w_i [1 + s e + 9/2 e^2 - 3/2 q] + a u(y).Jbar(y) + G.Jbar(y)
//     lambda_u(y) = sum_i gbar_i w_i rho(y) [s c_i + 9 e c_i - 3 u(y)] + a rho(y) Jbar(y)
//     dL/dnu     += sum_y [ sum_i gbar_i 18 w_i rho(y) e  - 6 rho(y) u(y).Jbar(y) ]
// (s = 18 nu and a = 1 - 6 nu carry all of the nu-dependence, Eq. ACM2.0nu). The
// dL/dnu sum is accumulated in FP64: per-block partials, then the block that
// finishes last adds them in a fixed order to a running total (deterministic).
//
// (Dbar, Jbar) of a step are pointwise in lambda+ and the state at t+1, which are
// the lambda and the state of the step before it in the backward sweep: the gather
// of step t writes (Dbar, Jbar) for step t-1 straight from its lambda_t and the
// state at t it already holds, so only the first step of the sweep runs the
// separate prep pass and only the last one writes lambda.
#include "dev_cache.h"
#include "launch.h"
#include "lwacm_core.cuh"
#include "tile_common.cuh"

namespace lwacm {
namespace {

constexpr int kAdjBlocks = 152 * 6;

// (Dbar, Jbar) from lambda+ and the state at t+1: four FP32 fields (three in 2D)
template <int Q>
__global__ void __launch_bounds__(256) k_adj_prep(const float *__restrict__ sn, const float *__restrict__ lam,
                                                  float *__restrict__ dj, long long fstride, long long N) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        const float rn = 1.f + sn[k];
        const float inv = 1.f / rn;
        const float lu = lam[fstride + k], lv = lam[2 * fstride + k];
        const float lw = Q == 19 ? lam[3 * fstride + k] : 0.f;
        const float un = sn[fstride + k], vn = sn[2 * fstride + k];
        const float wn = Q == 19 ? sn[3 * fstride + k] : 0.f;
        dj[k] = lam[k] - (lu * un + lv * vn + lw * wn) * inv;
        dj[fstride + k] = lu * inv;
        dj[2 * fstride + k] = lv * inv;
        if (Q == 19) dj[3 * fstride + k] = lw * inv;
    }
}

// lambda at t from (Dbar, Jbar) gathered at the downwind neighbours and the state
// at t, with the (Dbar, Jbar) fields staged in shared memory: a CTA of
// 32 x 8 threads takes an x-y tile of the domain and marches along z through a run
// of planes, keeping the planes z-1, z, z+1 of the tile plus a one-node frame in a
// ring of five shared-memory slots, the plane z+2 arriving by asynchronous copies
// while the plane z is computed (five slots: the slot a copy refills was last read
// two planes earlier, so one barrier per plane orders it). The state at t of the
// plane z+1 is loaded into registers while the plane z is computed.
constexpr int ATX = 32, ATY = 8, AZC = 8;
constexpr int AW = ATX + 2, AH = ATY + 2, APL = AW * AH, NSL = 5;

// With WALLS, a link whose receiver x + c lies beyond a walled face is the value the
// node itself takes for the bounced link -c (Eq. ACM2.0cccbb2): gbar = Dbar - c.Jbar
// of the node; the moving-wall term of Eq. ACM2.0ccccbb adds its nu-derivative.
// NEXT: write (Dbar, Jbar) of the next step of the sweep to `out` instead of lambda.
template <int Q, bool WALLS, bool NEXT>
__global__ void __launch_bounds__(ATX *ATY) k_adj_gather_tiled(const float *__restrict__ st,
                                                               const float *__restrict__ dj,
                                                               float *__restrict__ out, StepParams p, int ntx,
                                                               int nty, int nzc, double *__restrict__ nu_partial,
                                                               unsigned *__restrict__ done,
                                                               double *__restrict__ nu_total) {
    using L = Lat<Q>;
    constexpr int NF = Q == 19 ? 4 : 3;
    __shared__ float ring[NSL][NF][APL];
    const int tid = (int)threadIdx.x, tx = tid % ATX, ty = tid / ATX;
    const long long plane = (long long)p.nx * p.ny;
    double nu_acc = 0.0;  // FP64 over items; FP32 within an item's run of planes
    const long long nitems = (long long)ntx * nty * nzc;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = (int)(item % ntx), by = (int)((item / ntx) % nty), bz = (int)(item / ((long long)ntx * nty));
        const int x0 = bx * ATX, y0 = by * ATY, za = bz * AZC;
        const int zb = za + AZC < p.nz ? za + AZC : p.nz;
        // in-plane offsets of this thread's (at most two) tile + frame elements,
        // wrapped periodically once per item
        constexpr int NE = (APL + ATX * ATY - 1) / (ATX * ATY);
        long long off2[NE];
#pragma unroll
        for (int r = 0; r < NE; ++r) {
            const int e = tid + r * ATX * ATY;
            int gx = (x0 + e % AW - 1) % p.nx, gy = (y0 + e / AW - 1) % p.ny;
            if (gx < 0) gx += p.nx;
            if (gy < 0) gy += p.ny;
            off2[r] = (long long)gy * p.nx + gx;
        }
        // asynchronous copy of plane z (periodic) of the tile + frame into ring slot
        // (z - za + 1) % NSL
        auto slot_of = [&](int z) { return (z - za + 1) % NSL; };
        auto issue = [&](int z) {
            const int zl = z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z);
            const int slot = slot_of(z);
#pragma unroll
            for (int r = 0; r < NE; ++r) {
                const int e = tid + r * ATX * ATY;
                if (e < APL) {
                    const float *src = dj + (long long)zl * plane + off2[r];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const unsigned dst = (unsigned)__cvta_generic_to_shared(&ring[slot][f][e]);
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src + f * p.fstride)
                                     : "memory");
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        float nu_run = 0.f;
        const int x = x0 + tx, y = y0 + ty;
        const bool inside = x < p.nx && y < p.ny;
        const long long k0 = (long long)y * p.nx + x;
        // the state at t of plane za (then prefetched one plane ahead)
        float d = 0.f, u = 0.f, v = 0.f, w = 0.f;
        if (inside) {
            const long long k = (long long)za * plane + k0;
            d = st[k];
            u = st[p.fstride + k];
            v = st[2 * p.fstride + k];
            if (Q == 19) w = st[3 * p.fstride + k];
        }
        __syncthreads();  // the previous item's last reads are done
        issue(za - 1);
        issue(za);
        issue(za + 1);
        for (int z = za; z < zb; ++z) {
            // planes z-1, z, z+1 complete (z+2 may still be in flight)
            if (z + 2 <= zb) {
                issue(z + 2);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            float dn = 0.f, un = 0.f, vn = 0.f, wn = 0.f;
            if (inside && z + 1 < zb) {
                const long long k = (long long)(z + 1) * plane + k0;
                dn = st[k];
                un = st[p.fstride + k];
                vn = st[2 * p.fstride + k];
                if (Q == 19) wn = st[3 * p.fstride + k];
            }
            const int sm = slot_of(z - 1), s0 = slot_of(z), sp = slot_of(z + 1);
            if (inside) {
                const long long k = (long long)z * plane + k0;
                const float rho = 1.f + d;
                const float q = fmaf(u, u, fmaf(v, v, w * w));
                // weighted moments of gbar_i = Dbar + c_i . Jbar over the links:
                //   G0 = sum w gbar, G1 = sum w c gbar, G2 = sum w c c gbar, so that
                //   sum_i gbar_i dg_i/dd = (1 - 3/2 q) G0 + s u.G1 + 9/2 u.G2.u,
                //   sum_i gbar_i dg_i/du = rho (s G1 + 9 G2.u - 3 u G0),
                //   sum_i gbar_i dg_i/ds = rho u.G1
                float g0 = 0.f, g1x = 0.f, g1y = 0.f, g1z = 0.f;
                float gxx = 0.f, gyy = 0.f, gzz = 0.f, gxy = 0.f, gxz = 0.f, gyz = 0.f;
                float nu_wall = 0.f;  // sum over lid links of gbar * d(wall term)/dnu
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
                    const float wi = L::w(i);
                    const int slot = cz < 0 ? sm : (cz > 0 ? sp : s0);
                    const int e = (ty + 1 + cy) * AW + tx + 1 + cx;
                    float gb = ring[slot][0][e];
                    if (cx) gb = fmaf((float)cx, ring[slot][1][e], gb);
                    if (cy) gb = fmaf((float)cy, ring[slot][2][e], gb);
                    if (Q == 19 && cz) gb = fmaf((float)cz, ring[slot][3][e], gb);
                    if (WALLS && i > 0) {
                        const int xr = x + cx, yr = y + cy, zr = z + cz;
                        const bool out = (p.walled[0] && (xr < 0 || xr >= p.nx)) ||
                                         (p.walled[1] && (yr < 0 || yr >= p.ny)) ||
                                         (Q == 19 && p.walled[2] && (zr < 0 || zr >= p.nz));
                        if (out) {
                            const int os0 = s0, own0 = (ty + 1) * AW + tx + 1;
                            float b = ring[os0][0][own0];
                            if (cx) b = fmaf((float)-cx, ring[os0][1][own0], b);
                            if (cy) b = fmaf((float)-cy, ring[os0][2][own0], b);
                            if (Q == 19 && cz) b = fmaf((float)-cz, ring[os0][3][own0], b);
                            gb = b;
                            const int rl = p.lid_axis == 0 ? xr : (p.lid_axis == 1 ? yr : zr);
                            const int nl = p.lid_axis == 0 ? p.nx : (p.lid_axis == 1 ? p.ny : p.nz);
                            if (rl >= nl) {
                                // wall term w (36 nu rho0)(-c.u_w) of the bounced link
                                const float cu = cx * p.lid[0] + cy * p.lid[1] + cz * p.lid[2];
                                nu_wall = fmaf(gb, -wi * cu, nu_wall);
                            }
                        }
                    }
                    g0 = fmaf(wi, gb, g0);
                    if (cx) g1x = fmaf(wi * cx, gb, g1x);
                    if (cy) g1y = fmaf(wi * cy, gb, g1y);
                    if (cz) g1z = fmaf(wi * cz, gb, g1z);
                    if (cx) gxx = fmaf(wi, gb, gxx);
                    if (cy) gyy = fmaf(wi, gb, gyy);
                    if (cz) gzz = fmaf(wi, gb, gzz);
                    if (cx && cy) gxy = fmaf(wi * cx * cy, gb, gxy);
                    if (cx && cz) gxz = fmaf(wi * cx * cz, gb, gxz);
                    if (cy && cz) gyz = fmaf(wi * cy * cz, gb, gyz);
                }
                const float hx = fmaf(gxx, u, fmaf(gxy, v, gxz * w));  // G2 . u
                const float hy = fmaf(gxy, u, fmaf(gyy, v, gyz * w));
                const float hz = fmaf(gxz, u, fmaf(gyz, v, gzz * w));
                const float uG1 = fmaf(u, g1x, fmaf(v, g1y, w * g1z));
                const float uG2u = fmaf(u, hx, fmaf(v, hy, w * hz));
                float ld = fmaf(4.5f, uG2u, fmaf(p.s, uG1, g0 * fmaf(-1.5f, q, 1.f)));
                const float m3 = -3.f * g0;
                float lu = rho * fmaf(p.s, g1x, fmaf(9.f, hx, m3 * u));
                float lv = rho * fmaf(p.s, g1y, fmaf(9.f, hy, m3 * v));
                float lw = Q == 19 ? rho * fmaf(p.s, g1z, fmaf(9.f, hz, m3 * w)) : 0.f;
                const float ln = rho * uG1;
                const int own = (ty + 1) * AW + tx + 1, os = s0;
                const float jx = ring[os][1][own], jy = ring[os][2][own];
                const float jz = Q == 19 ? ring[os][3][own] : 0.f;
                const float ju = u * jx + v * jy + w * jz;
                ld = fmaf(p.a, ju, ld);
                if (p.has_force) ld += p.force[0] * jx + p.force[1] * jy + p.force[2] * jz;
                lu = fmaf(p.a * rho, jx, lu);
                lv = fmaf(p.a * rho, jy, lv);
                lw = fmaf(p.a * rho, jz, lw);
                if (NEXT) {  // the prep of the next step: this node's state at t is its state at t+1
                    const float inv = 1.f / rho;
                    out[k] = ld - (lu * u + lv * v + lw * w) * inv;
                    out[p.fstride + k] = lu * inv;
                    out[2 * p.fstride + k] = lv * inv;
                    if (Q == 19) out[3 * p.fstride + k] = lw * inv;
                } else {
                    out[k] = ld;
                    out[p.fstride + k] = lu;
                    out[2 * p.fstride + k] = lv;
                    if (Q == 19) out[3 * p.fstride + k] = lw;
                }
                nu_run += fmaf(18.f, ln, -6.f * rho * ju);
                if (WALLS) nu_run = fmaf(18.f * p.wallc / p.s, nu_wall, nu_run);  // 36 rho0 = wallc / nu
            }
            d = dn;
            u = un;
            v = vn;
            w = wn;
        }
        nu_acc += (double)nu_run;
    }
    __shared__ double sh[ATX * ATY];
    sh[tid] = nu_acc;
    __syncthreads();
    for (int off = ATX * ATY / 2; off > 0; off >>= 1) {
        if (tid < off) sh[tid] += sh[tid + off];
        __syncthreads();
    }
    // the block that finishes last adds the partials in a fixed order
    __shared__ bool last;
    if (tid == 0) {
        nu_partial[blockIdx.x] = sh[0];
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    double a = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += ATX * ATY) a += __ldcg(nu_partial + b);
    sh[tid] = a;
    __syncthreads();
    for (int off = ATX * ATY / 2; off > 0; off >>= 1) {
        if (tid < off) sh[tid] += sh[tid + off];
        __syncthreads();
    }
    if (tid == 0) {
        *nu_total += sh[0];
        *done = 0u;  // ready for the next step (stream-ordered)
    }
}

// ---- row-tiled gather (D3Q19, periodic, nx = 128 NH, ny a multiple of 8) --------
// The same derivative as k_adj_gather_tiled, organised like the forward half-row
// kernel: a CTA takes a column of 8 full rows (NH warps per row, four nodes per
// lane) and marches along z; the planes of (Dbar, Jbar) it reads, 10 rows each
// (the column and one row either side), arrive by 1-D bulk copies (mbarrier
// completion) in a ring of four slots: planes z-1, z, z+1 are read while z+2 is in
// flight. Links are taken in pairs (c, -c), gbar+ = Dbar(y+c) + c.Jbar(y+c) and
// gbar- = Dbar(y-c) - c.Jbar(y-c), and enter the moments through their sum
// S = gbar+ + gbar- and difference D = gbar+ - gbar-:
//   G0 += w S,  G1_a += w c_a D,  G2_ab += w c_a c_b S.
// The state at t of the node is read straight from global memory (coalesced).
namespace arow {

constexpr int ROWS = 8, TROWS = ROWS + 2, NSLOT = 4;

template <int NH>
struct RG {
    static constexpr int NX = 128 * NH, NTH = ROWS * NH * 32;
    static constexpr int PLANE = 4 * TROWS * NX;  // floats per slot: 4 fields x 10 rows
    static constexpr size_t BYTES = (size_t)NSLOT * PLANE * 4 + 64;
};

struct RowParams {
    int nx, ny, nz, ycols, zc, nitems;
    long long fstride;
    float s, a;       // 18 nu, 1 - 6 nu
    float g[3];       // constant acceleration (Eq. force) or 0
    int *err;
};

// one plane of the 4 (Dbar, Jbar) fields, rows y0-1 .. y0+8 (periodic in y and z)
template <int NH>
__device__ __forceinline__ void issue_plane(const float *dj, const RowParams &p, int col, int z, float *slot,
                                            uint64_t *bar) {
    using namespace lwacm::tile;
    constexpr int NX = RG<NH>::NX;
    const int zl = z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z);
    const int y0 = col * ROWS;
    const long long plane = (long long)NX * p.ny;
    mbar_expect_tx(bar, (uint32_t)(RG<NH>::PLANE * 4));
    constexpr uint32_t rb = NX * 4;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const float *src = dj + f * p.fstride + (long long)zl * plane;
        float *dst = slot + f * TROWS * NX;
        if (y0 >= 1 && y0 + ROWS < p.ny) {
            bulk_g2s(dst, src + (long long)(y0 - 1) * NX, TROWS * rb, bar);
        } else {
            const int yb = y0 - 1 < 0 ? y0 - 1 + p.ny : y0 - 1;
            const int yt = y0 + ROWS >= p.ny ? y0 + ROWS - p.ny : y0 + ROWS;
            bulk_g2s(dst, src + (long long)yb * NX, rb, bar);
            bulk_g2s(dst + NX, src + (long long)y0 * NX, ROWS * rb, bar);
            bulk_g2s(dst + (TROWS - 1) * NX, src + (long long)yt * NX, rb, bar);
        }
    }
}

// six consecutive values of a staged row, x0-1 .. x0+4 (periodic in x): v[1..4] are
// the lane's own four nodes
template <int NX>
__device__ __forceinline__ void row6(const float *r, int x0, float (&v)[6]) {
    const float4 m = *reinterpret_cast<const float4 *>(r + x0);
    v[0] = r[(x0 + NX - 1) & (NX - 1)];
    v[1] = m.x;
    v[2] = m.y;
    v[3] = m.z;
    v[4] = m.w;
    v[5] = r[(x0 + 4) & (NX - 1)];
}
__device__ __forceinline__ void row4(const float *r, int x0, float (&v)[4]) {
    const float4 m = *reinterpret_cast<const float4 *>(r + x0);
    v[0] = m.x;
    v[1] = m.y;
    v[2] = m.z;
    v[3] = m.w;
}

struct Mom {
    float g0[4], g1[3][4], g2[6][4];  // G0, G1 (x, y, z), G2 (xx, yy, zz, xy, xz, yz)
};
// accumulate the pair (c, -c) of weight w from gbar+ / gbar- of the four nodes
template <int CX, int CY, int CZ>
__device__ __forceinline__ void pair_moments(Mom &m, float w, const float (&gp)[4], const float (&gm)[4]) {
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const float S = gp[n] + gm[n], D = gp[n] - gm[n];
        m.g0[n] = fmaf(w, S, m.g0[n]);
        if (CX) m.g1[0][n] = fmaf(w * CX, D, m.g1[0][n]);
        if (CY) m.g1[1][n] = fmaf(w * CY, D, m.g1[1][n]);
        if (CZ) m.g1[2][n] = fmaf(w * CZ, D, m.g1[2][n]);
        if (CX) m.g2[0][n] = fmaf(w, S, m.g2[0][n]);
        if (CY) m.g2[1][n] = fmaf(w, S, m.g2[1][n]);
        if (CZ) m.g2[2][n] = fmaf(w, S, m.g2[2][n]);
        if (CX && CY) m.g2[3][n] = fmaf(w * CX * CY, S, m.g2[3][n]);
        if (CX && CZ) m.g2[4][n] = fmaf(w * CX * CZ, S, m.g2[4][n]);
        if (CY && CZ) m.g2[5][n] = fmaf(w * CY * CZ, S, m.g2[5][n]);
    }
}

// the moments of one node quadruple from the three staged planes (slots sm, s0, sp
// hold planes z-1, z, z+1), row rs of the slot (rs = row + 1)
template <int NH>
__device__ __forceinline__ void gather(Mom &m, const float *sm, const float *s0, const float *sp, int rs, int x0,
                                       float (&own)[4][4]) {
    constexpr int NX = RG<NH>::NX, FS = TROWS * NX;  // field stride in a slot
    constexpr float WA = 1.f / 18.f, WD = 1.f / 36.f;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        m.g0[n] = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) m.g1[a][n] = 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) m.g2[a][n] = 0.f;
    }
    {  // plane z, own row: the rest link, (1,0,0), and the node's own (Dbar, Jbar)
        float D[6], Jx[6];
        row6<NX>(s0 + rs * NX, x0, D);
        row6<NX>(s0 + FS + rs * NX, x0, Jx);
        row4(s0 + 2 * FS + rs * NX, x0, own[2]);
        row4(s0 + 3 * FS + rs * NX, x0, own[3]);
        float gp[4], gm[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            own[0][n] = D[n + 1];
            own[1][n] = Jx[n + 1];
            m.g0[n] = (1.f / 3.f) * D[n + 1];
            gp[n] = D[n + 2] + Jx[n + 2];
            gm[n] = D[n] - Jx[n];
        }
        pair_moments<1, 0, 0>(m, WA, gp, gm);
    }
    {  // plane z, rows rs -+ 1: (0,1,0), (1,1,0), (1,-1,0)
        float Du[6], Xu[6], Yu[6], Dd[6], Xd[6], Yd[6];
        row6<NX>(s0 + (rs + 1) * NX, x0, Du);
        row6<NX>(s0 + FS + (rs + 1) * NX, x0, Xu);
        row6<NX>(s0 + 2 * FS + (rs + 1) * NX, x0, Yu);
        row6<NX>(s0 + (rs - 1) * NX, x0, Dd);
        row6<NX>(s0 + FS + (rs - 1) * NX, x0, Xd);
        row6<NX>(s0 + 2 * FS + (rs - 1) * NX, x0, Yd);
        float gp[4], gm[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            gp[n] = Du[n + 1] + Yu[n + 1];
            gm[n] = Dd[n + 1] - Yd[n + 1];
        }
        pair_moments<0, 1, 0>(m, WA, gp, gm);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            gp[n] = Du[n + 2] + Xu[n + 2] + Yu[n + 2];  // (1,1,0) from (x+1, y+1)
            gm[n] = Dd[n] - Xd[n] - Yd[n];              // (-1,-1,0) from (x-1, y-1)
        }
        pair_moments<1, 1, 0>(m, WD, gp, gm);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            gp[n] = Dd[n + 2] + Xd[n + 2] - Yd[n + 2];  // (1,-1,0) from (x+1, y-1)
            gm[n] = Du[n] - Xu[n] + Yu[n];              // (-1,1,0) from (x-1, y+1)
        }
        pair_moments<1, -1, 0>(m, WD, gp, gm);
    }
    {  // planes z -+ 1, own row: (0,0,1), (1,0,1), (1,0,-1)
        float Da[6], Xa[6], Za[6], Db[6], Xb[6], Zb[6];
        row6<NX>(sp + rs * NX, x0, Da);
        row6<NX>(sp + FS + rs * NX, x0, Xa);
        row6<NX>(sp + 3 * FS + rs * NX, x0, Za);
        row6<NX>(sm + rs * NX, x0, Db);
        row6<NX>(sm + FS + rs * NX, x0, Xb);
        row6<NX>(sm + 3 * FS + rs * NX, x0, Zb);
        float gp[4], gm[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            gp[n] = Da[n + 1] + Za[n + 1];
            gm[n] = Db[n + 1] - Zb[n + 1];
        }
        pair_moments<0, 0, 1>(m, WA, gp, gm);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            gp[n] = Da[n + 2] + Xa[n + 2] + Za[n + 2];  // (1,0,1) from (x+1, z+1)
            gm[n] = Db[n] - Xb[n] - Zb[n];              // (-1,0,-1) from (x-1, z-1)
        }
        pair_moments<1, 0, 1>(m, WD, gp, gm);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            gp[n] = Db[n + 2] + Xb[n + 2] - Zb[n + 2];  // (1,0,-1) from (x+1, z-1)
            gm[n] = Da[n] - Xa[n] + Za[n];              // (-1,0,1) from (x-1, z+1)
        }
        pair_moments<1, 0, -1>(m, WD, gp, gm);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // (0,1,1) and (0,1,-1): rows rs -+ 1 of planes z -+ 1
        const float *pu = k == 0 ? sp : sm, *pd = k == 0 ? sm : sp;  // c = (0,1,+-1): up row in plane z+-1
        float Du[4], Yu[4], Zu[4], Dd[4], Yd[4], Zd[4];
        row4(pu + (rs + 1) * NX, x0, Du);
        row4(pu + 2 * FS + (rs + 1) * NX, x0, Yu);
        row4(pu + 3 * FS + (rs + 1) * NX, x0, Zu);
        row4(pd + (rs - 1) * NX, x0, Dd);
        row4(pd + 2 * FS + (rs - 1) * NX, x0, Yd);
        row4(pd + 3 * FS + (rs - 1) * NX, x0, Zd);
        const float cz = k == 0 ? 1.f : -1.f;
        float gp[4], gm[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            gp[n] = fmaf(cz, Zu[n], Du[n] + Yu[n]);
            gm[n] = fmaf(-cz, Zd[n], Dd[n] - Yd[n]);
        }
        if (k == 0)
            pair_moments<0, 1, 1>(m, WD, gp, gm);
        else
            pair_moments<0, 1, -1>(m, WD, gp, gm);
    }
}

template <int NH, bool NEXT>
__global__ void __launch_bounds__(RG<NH>::NTH, 2 / NH) k_adj_rows(const float *__restrict__ st,
                                                                 const float *__restrict__ dj,
                                                                 float *__restrict__ out, RowParams p,
                                                                 double *__restrict__ nu_partial,
                                                                 unsigned *__restrict__ done,
                                                                 double *__restrict__ nu_total) {
    using namespace lwacm::tile;
    constexpr int NX = RG<NH>::NX, PLANE = RG<NH>::PLANE, NTH = RG<NH>::NTH;
    extern __shared__ float4 smem4[];
    float *ring = reinterpret_cast<float *>(smem4);
    uint64_t *bars = reinterpret_cast<uint64_t *>(ring + NSLOT * PLANE);
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row = NH == 2 ? warp >> 1 : warp, half = NH == 2 ? (warp & 1) : 0;
    const int x0 = half * 128 + lane * 4;
    const bool producer = tid == 0;
    __shared__ int failed;
    if (tid == 0) {
        failed = 0;
        for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long long plane = (long long)NX * p.ny;
    double nu_acc = 0.0;
    unsigned ic = 0;  // planes issued so far: plane number k sits in slot k % 4, mbarrier phase k / 4
    auto wait_k = [&](unsigned k) { return mbar_wait(&bars[k % NSLOT], (k / NSLOT) & 1u); };
    for (int item = blockIdx.x; item < p.nitems; item += gridDim.x) {
        const int col = item % p.ycols, ch = item / p.ycols;
        const int za = ch * p.zc, zb = za + p.zc < p.nz ? za + p.zc : p.nz;
        const unsigned k0 = ic;
        __syncthreads();  // the previous item's reads of every slot are done
        if (producer)
            for (int j = 0; j < 3; ++j)
                issue_plane<NH>(dj, p, col, za - 1 + j, ring + ((k0 + j) % NSLOT) * PLANE, &bars[(k0 + j) % NSLOT]);
        ic = k0 + (unsigned)(zb - za) + 2;
        bool ok = wait_k(k0) && wait_k(k0 + 1);
        float nu_run = 0.f;
        const long long k_row = (long long)(col * ROWS + row) * NX + x0;
        for (int z = za; z < zb; ++z) {
            const unsigned kz = k0 + (unsigned)(z - za) + 1;  // plane z
            // the state at t of the lane's four nodes, requested before the waits below
            const long long k = (long long)z * plane + k_row;
            const float4 d4 = *reinterpret_cast<const float4 *>(st + k);
            const float4 u4 = *reinterpret_cast<const float4 *>(st + p.fstride + k);
            const float4 v4 = *reinterpret_cast<const float4 *>(st + 2 * p.fstride + k);
            const float4 w4 = *reinterpret_cast<const float4 *>(st + 3 * p.fstride + k);
            ok = ok && wait_k(kz + 1);
            if (!ok) failed = 1;
            __syncthreads();  // everyone is past plane z-1: the slot of plane z-2 is free
            if (failed) {
                if (producer) {  // plane z+1 is the only copy that may still be in flight
                    atomicExch(p.err, 1);
                    wait_k(kz + 1);
                }
                return;
            }
            if (producer && z + 2 <= zb) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_plane<NH>(dj, p, col, z + 2, ring + ((kz + 2) % NSLOT) * PLANE, &bars[(kz + 2) % NSLOT]);
            }
            Mom m;
            float own[4][4];
            gather<NH>(m, ring + ((kz - 1) % NSLOT) * PLANE, ring + (kz % NSLOT) * PLANE,
                       ring + ((kz + 1) % NSLOT) * PLANE, row + 1, x0, own);
            const float dd[4] = {d4.x, d4.y, d4.z, d4.w}, uu[4] = {u4.x, u4.y, u4.z, u4.w};
            const float vv[4] = {v4.x, v4.y, v4.z, v4.w}, ww[4] = {w4.x, w4.y, w4.z, w4.w};
            float o[4][4];
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const float u = uu[n], v = vv[n], w = ww[n], rho = 1.f + dd[n];
                const float q = fmaf(u, u, fmaf(v, v, w * w));
                const float hx = fmaf(m.g2[0][n], u, fmaf(m.g2[3][n], v, m.g2[4][n] * w));  // G2 . u
                const float hy = fmaf(m.g2[3][n], u, fmaf(m.g2[1][n], v, m.g2[5][n] * w));
                const float hz = fmaf(m.g2[4][n], u, fmaf(m.g2[5][n], v, m.g2[2][n] * w));
                const float uG1 = fmaf(u, m.g1[0][n], fmaf(v, m.g1[1][n], w * m.g1[2][n]));
                const float uG2u = fmaf(u, hx, fmaf(v, hy, w * hz));
                float ld = fmaf(4.5f, uG2u, fmaf(p.s, uG1, m.g0[n] * fmaf(-1.5f, q, 1.f)));
                const float m3 = -3.f * m.g0[n];
                float lu = rho * fmaf(p.s, m.g1[0][n], fmaf(9.f, hx, m3 * u));
                float lv = rho * fmaf(p.s, m.g1[1][n], fmaf(9.f, hy, m3 * v));
                float lw = rho * fmaf(p.s, m.g1[2][n], fmaf(9.f, hz, m3 * w));
                const float jx = own[1][n], jy = own[2][n], jz = own[3][n];
                const float ju = fmaf(u, jx, fmaf(v, jy, w * jz));
                ld = fmaf(p.a, ju, ld);
                ld = fmaf(p.g[0], jx, fmaf(p.g[1], jy, fmaf(p.g[2], jz, ld)));  // Eq. force (g = 0 without)
                const float ar = p.a * rho;
                lu = fmaf(ar, jx, lu);
                lv = fmaf(ar, jy, lv);
                lw = fmaf(ar, jz, lw);
                if (NEXT) {  // (Dbar, Jbar) of the next step of the sweep
                    const float inv = lwacm::tile::rcp_rn(rho);  // 1 / rho, correctly rounded, no branch
                    o[0][n] = ld - (lu * u + lv * v + lw * w) * inv;
                    o[1][n] = lu * inv;
                    o[2][n] = lv * inv;
                    o[3][n] = lw * inv;
                } else {
                    o[0][n] = ld;
                    o[1][n] = lu;
                    o[2][n] = lv;
                    o[3][n] = lw;
                }
                nu_run += fmaf(18.f, rho * uG1, -6.f * rho * ju);
            }
#pragma unroll
            for (int f = 0; f < 4; ++f)
                *reinterpret_cast<float4 *>(out + f * p.fstride + k) = make_float4(o[f][0], o[f][1], o[f][2], o[f][3]);
        }
        nu_acc += (double)nu_run;
    }
    // dL/dnu: block sum, then the block that finishes last adds the partials in order
    __shared__ double sh[NTH];
    sh[tid] = nu_acc;
    __syncthreads();
    for (int off = NTH / 2; off > 0; off >>= 1) {
        if (tid < off) sh[tid] += sh[tid + off];
        __syncthreads();
    }
    __shared__ bool last;
    if (tid == 0) {
        nu_partial[blockIdx.x] = sh[0];
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    double a = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += NTH) a += __ldcg(nu_partial + b);
    sh[tid] = a;
    __syncthreads();
    for (int off = NTH / 2; off > 0; off >>= 1) {
        if (tid < off) sh[tid] += sh[tid + off];
        __syncthreads();
    }
    if (tid == 0) {
        *nu_total += sh[0];
        *done = 0u;
    }
}

template <int NH, bool NEXT>
int rows_ctas() {
    static DevSlots slots;
    return per_device(slots, [] {
        if (cudaFuncSetAttribute(k_adj_rows<NH, NEXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)RG<NH>::BYTES) != cudaSuccess)
            return -1;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_rows<NH, NEXT>, RG<NH>::NTH, RG<NH>::BYTES) !=
                cudaSuccess ||
            nb < 1)
            return -1;
        return nb * device_sms();
    });
}

template <int NH, bool NEXT>
cudaError_t launch_rows(const float *state_t, const float *dj, float *out, const StepParams &sp, double *part,
                        unsigned *done, double *total, cudaStream_t st) {
    const int ctas = rows_ctas<NH, NEXT>();
    if (ctas < 1) return cudaErrorNotSupported;
    RowParams p;
    p.nx = sp.nx;
    p.ny = sp.ny;
    p.nz = sp.nz;
    p.ycols = sp.ny / ROWS;
    // z-chunks: the run length that minimises the slowest CTA's work, counted as its
    // number of items times (planes per item + the two extra planes an item stages)
    int zc = sp.nz;
    double best = 1e300;
    for (int c = sp.nz < 4 ? sp.nz : 4; c <= sp.nz; ++c) {
        const long long items = (long long)p.ycols * ((sp.nz + c - 1) / c);
        const double t = (double)((items + ctas - 1) / ctas) * (c + 2.0);
        if (t < best - 1e-9) {
            best = t;
            zc = c;
        }
    }
    p.zc = zc;
    p.nitems = p.ycols * ((sp.nz + zc - 1) / zc);
    p.fstride = sp.fstride;
    p.s = sp.s;
    p.a = sp.a;
    for (int c = 0; c < 3; ++c) p.g[c] = sp.has_force ? sp.force[c] : 0.f;
    p.err = sp.err;
    int grid = ctas < p.nitems ? ctas : p.nitems;
    if (grid > kAdjBlocks) grid = kAdjBlocks;
    k_adj_rows<NH, NEXT><<<grid, RG<NH>::NTH, RG<NH>::BYTES, st>>>(state_t, dj, out, p, part, done, total);
    return cudaGetLastError();
}

}  // namespace arow

// the row-tiled gather serves D3Q19 periodic domains with 128- or 256-node rows
bool rows_supported(const StepParams &p) {
    return p.nz >= 1 && (p.nx == 128 || p.nx == 256) && p.ny >= 8 && p.ny % 8 == 0 && !p.walled[0] &&
           !p.walled[1] && !p.walled[2] && p.err && p.fstride % 4 == 0 && !p.gfield;
}

}  // namespace

int adjoint_partials() { return kAdjBlocks; }

template <int Q, bool WALLS>
static void gather(bool next, int grid, const float *state_t, const float *dj, float *out, const StepParams &p,
                   int ntx, int nty, int nzc, double *part, unsigned *done, double *total, cudaStream_t st) {
    if (next)
        k_adj_gather_tiled<Q, WALLS, true>
            <<<grid, ATX * ATY, 0, st>>>(state_t, dj, out, p, ntx, nty, nzc, part, done, total);
    else
        k_adj_gather_tiled<Q, WALLS, false>
            <<<grid, ATX * ATY, 0, st>>>(state_t, dj, out, p, ntx, nty, nzc, part, done, total);
}

cudaError_t launch_adjoint_step(int Q, const float *state_t, const float *state_t1, const float *lam_t1,
                                float *dj, float *dj_next, float *lam_t, const StepParams &p, double *nu_partial,
                                unsigned *done, double *nu_total, cudaStream_t st) {
    // tiled gather: x-y tiles of 32 x 8, z-runs of 16 planes; every CTA writes one
    // partial (the grid never exceeds the partials buffer)
    const int ntx = (p.nx + ATX - 1) / ATX, nty = (p.ny + ATY - 1) / ATY, nzc = (p.nz + AZC - 1) / AZC;
    const long long items = (long long)ntx * nty * nzc;
    const int grid = (int)(items < kAdjBlocks ? items : kAdjBlocks);
    const bool walls = p.walled[0] || p.walled[1] || p.walled[2];
    const bool next = dj_next != nullptr;
    float *out = next ? dj_next : lam_t;
    if (Q == 9) {
        if (lam_t1) k_adj_prep<9><<<kAdjBlocks, 256, 0, st>>>(state_t1, lam_t1, dj, p.fstride, p.N);
        if (walls)
            gather<9, true>(next, grid, state_t, dj, out, p, ntx, nty, nzc, nu_partial, done, nu_total, st);
        else
            gather<9, false>(next, grid, state_t, dj, out, p, ntx, nty, nzc, nu_partial, done, nu_total, st);
    } else {
        if (lam_t1) k_adj_prep<19><<<kAdjBlocks, 256, 0, st>>>(state_t1, lam_t1, dj, p.fstride, p.N);
        if (rows_supported(p)) {
            if (p.nx == 256)
                return next ? arow::launch_rows<2, true>(state_t, dj, out, p, nu_partial, done, nu_total, st)
                            : arow::launch_rows<2, false>(state_t, dj, out, p, nu_partial, done, nu_total, st);
            return next ? arow::launch_rows<1, true>(state_t, dj, out, p, nu_partial, done, nu_total, st)
                        : arow::launch_rows<1, false>(state_t, dj, out, p, nu_partial, done, nu_total, st);
        }
        if (walls)
            gather<19, true>(next, grid, state_t, dj, out, p, ntx, nty, nzc, nu_partial, done, nu_total, st);
        else
            gather<19, false>(next, grid, state_t, dj, out, p, ntx, nty, nzc, nu_partial, done, nu_total, st);
    }
    return cudaGetLastError();
}

}  // namespace lwacm
