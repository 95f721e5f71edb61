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
#include "launch.h"
#include "lwacm_core.cuh"

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
        if (walls)
            gather<19, true>(next, grid, state_t, dj, out, p, ntx, nty, nzc, nu_partial, done, nu_total, st);
        else
            gather<19, false>(next, grid, state_t, dj, out, p, ntx, nty, nzc, nu_partial, done, nu_total, st);
    }
    return cudaGetLastError();
}

}  // namespace lwacm
