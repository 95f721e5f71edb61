// Adjoint (reverse-mode derivative) of one LW-ACM step in the moment form, for
// periodic domains with optional forcing.
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
// dL/dnu sum is accumulated in FP64: per-block partials, then one block adds them
// in a fixed order to a running total (deterministic).
#include "launch.h"
#include "lwacm_core.cuh"

namespace lwacm {
namespace {

constexpr int kAdjBlocks = 152 * 4;

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

// lambda at t from (Dbar, Jbar) gathered at the downwind neighbours and the state at t
template <int Q>
__global__ void __launch_bounds__(256) k_adj_gather(const float *__restrict__ st, const float *__restrict__ dj,
                                                    float *__restrict__ lam_out, StepParams p,
                                                    double *__restrict__ nu_partial) {
    using L = Lat<Q>;
    double nu_acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < p.N;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % p.nx);
        const long long r = k / p.nx;
        const int y = (int)(r % p.ny);
        const int z = (int)(r / p.ny);
        const float d = st[k], u = st[p.fstride + k], v = st[2 * p.fstride + k];
        const float w = Q == 19 ? st[3 * p.fstride + k] : 0.f;
        const float rho = 1.f + d;
        const float q = fmaf(u, u, fmaf(v, v, w * w));
        float ld = 0.f, lu = 0.f, lv = 0.f, lw = 0.f, ln = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
            int rx = x + cx, ry = y + cy, rz = z + cz;
            rx = rx < 0 ? rx + p.nx : (rx >= p.nx ? rx - p.nx : rx);
            ry = ry < 0 ? ry + p.ny : (ry >= p.ny ? ry - p.ny : ry);
            rz = rz < 0 ? rz + p.nz : (rz >= p.nz ? rz - p.nz : rz);
            const long long kr = ((long long)rz * p.ny + ry) * p.nx + rx;
            float gb = __ldg(dj + kr);  // gbar_i = Dbar + c_i . Jbar at y + c_i
            if (cx) gb = fmaf((float)cx, __ldg(dj + p.fstride + kr), gb);
            if (cy) gb = fmaf((float)cy, __ldg(dj + 2 * p.fstride + kr), gb);
            if (Q == 19 && cz) gb = fmaf((float)cz, __ldg(dj + 3 * p.fstride + kr), gb);
            const float e = cx * u + cy * v + cz * w;
            const float wg = L::w(i) * gb;
            // dg/dd = w [1 + s e + 9/2 e^2 - 3/2 q]
            ld = fmaf(wg, 1.f + fmaf(e, fmaf(4.5f, e, p.s), -1.5f * q), ld);
            // dg/du = w rho [s c + 9 e c - 3 u]
            const float cc = rho * (p.s + 9.f * e);
            const float m3 = -3.f * rho;
            lu = fmaf(wg, fmaf(cc, (float)cx, m3 * u), lu);
            lv = fmaf(wg, fmaf(cc, (float)cy, m3 * v), lv);
            if (Q == 19) lw = fmaf(wg, fmaf(cc, (float)cz, m3 * w), lw);
            ln = fmaf(wg, rho * e, ln);  // dg/ds = w rho e; ds/dnu = 18
        }
        const float jx = __ldg(dj + p.fstride + k), jy = __ldg(dj + 2 * p.fstride + k);
        const float jz = Q == 19 ? __ldg(dj + 3 * p.fstride + k) : 0.f;
        const float ju = u * jx + v * jy + w * jz;
        // post-combine a rho u (and forcing rho G): d/dd and d/du
        ld = fmaf(p.a, ju, ld);
        if (p.has_force) ld += p.force[0] * jx + p.force[1] * jy + p.force[2] * jz;
        lu = fmaf(p.a * rho, jx, lu);
        lv = fmaf(p.a * rho, jy, lv);
        lw = fmaf(p.a * rho, jz, lw);
        lam_out[k] = ld;
        lam_out[p.fstride + k] = lu;
        lam_out[2 * p.fstride + k] = lv;
        if (Q == 19) lam_out[3 * p.fstride + k] = lw;
        nu_acc += 18.0 * (double)ln - 6.0 * (double)rho * (double)ju;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = nu_acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) nu_partial[blockIdx.x] = sh[0];
}

// total += sum of the partials, in a fixed order
__global__ void k_adj_nu_sum(const double *__restrict__ partial, int n, double *__restrict__ total) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) a += partial[b];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total += sh[0];
}

}  // namespace

int adjoint_partials() { return kAdjBlocks; }

cudaError_t launch_adjoint_step(int Q, const float *state_t, const float *state_t1, const float *lam_t1,
                                float *dj, float *lam_t, const StepParams &p, double *nu_partial,
                                double *nu_total, cudaStream_t st) {
    if (Q == 9) {
        k_adj_prep<9><<<kAdjBlocks, 256, 0, st>>>(state_t1, lam_t1, dj, p.fstride, p.N);
        k_adj_gather<9><<<kAdjBlocks, 256, 0, st>>>(state_t, dj, lam_t, p, nu_partial);
    } else {
        k_adj_prep<19><<<kAdjBlocks, 256, 0, st>>>(state_t1, lam_t1, dj, p.fstride, p.N);
        k_adj_gather<19><<<kAdjBlocks, 256, 0, st>>>(state_t, dj, lam_t, p, nu_partial);
    }
    k_adj_nu_sum<<<1, 256, 0, st>>>(nu_partial, kAdjBlocks, nu_total);
    return cudaGetLastError();
}

}  // namespace lwacm
