// Device-side definitions shared by the LW-ACM kernels: lattice tables, storage
// conversions, per-launch parameters and the moment-form link term.
//
// Moment form of Eq. ACM2.0 used by every kernel. With rho = 1 + d, a = 2(omega-1)/omega
// = 1 - 6 nu (Eq. ACM2.0nu) and s = 3(1 - a) = 18 nu, the pre-combined value of
// Eq. ACM2.0b(a), f*_i = f^(e)_i - a f^(e,o)_i, minus its constant part w_i is
//
//     g_i(y) = w_i [ d(y) + rho(y) ( s e + 9/2 e^2 - 3/2 |u(y)|^2 ) ],   e = c_i . u(y)
//
// (f^(e,o)_i = 3 w_i rho c_i.u is the odd part of Eq. d2q9_equilibrium_compact,
// Eq. feqo). Streaming (Eq. ACM2.0b(b)) takes g_i from x - c_i, and the post-combine
// (Eq. ACM2.0b(c)) adds a f^(e,o)_i(x), whose zeroth moment vanishes and whose
// first moment is a rho(x) u(x). Since sum_i w_i = 1 and sum_i w_i c_i = 0:
//
//     d+(x) = sum_i g_i(x - c_i)
//     j+(x) = a rho(x) u(x) + sum_i c_i g_i(x - c_i)     [+ rho(x) g, Eq. force]
//     u+(x) = j+(x) / (1 + d+(x))                          (moments, Section 2.1)
//
// Walls (Eq. ACM2.0cccbb2 with Eq. ACM2.0ccccbb): when x - c_i lies beyond a wall,
// g_i(x - c_i) is replaced by g_BB(i)(x) + 36 nu w_i rho0 (c_i . u_w); 36 nu = 2 b * 3
// with b = 2/omega - 1 = 6 nu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lwacm {

// ---- lattices ---------------------------------------------------------------
// Link order on the device: rest, then links in +/- pairs (2k-1, 2k). The paper
// fixes no D3Q19 order and sums are order-independent up to rounding.
template <int Q>
struct Lat;

template <>
struct Lat<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return t[i][a];
    }
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 4.f / 9.f : (i <= 4 ? 1.f / 9.f : 1.f / 36.f);
    }
};

template <>
struct Lat<19> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
                                  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 1.f / 3.f : (i <= 6 ? 1.f / 18.f : 1.f / 36.f);
    }
};

// opposite link: pairs (2k-1, 2k)
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// ---- storage ----------------------------------------------------------------
__device__ __forceinline__ float ldf(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ldf(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ldf(const double *p) { return (float)__ldg(p); }

__device__ __forceinline__ void stf(float *p, float v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void stf(__half *p, float v) { *p = __float2half_rn(v); }

// ---- parameters ---------------------------------------------------------------
enum Bc { BC_PERIODIC = 0, BC_CAVITY = 1, BC_CHANNEL = 2 };

struct StepParams {
    int nx, ny, nz;
    int bc;
    long long N;        // nx*ny*nz
    long long fstride;  // elements between consecutive fields of one buffer
    float s;            // 18 nu
    float a;            // 1 - 6 nu = 2(omega-1)/omega
    float am1;          // a - 1 = -6 nu (rounded from the exact value, not from a)
    float wallc;        // 36 nu rho0 (moving-wall coefficient, times w_i c_i.u_w)
    float lid[3];       // u_w of the moving wall
    float force[3];     // g of Eq. force
    int has_force;
    const float *gfield;  // per-node g of Eq. force (D FP32 fields, stride fstride) or null
    float sdelta;         // 18 (nu_p - nu): pressure update relaxed with omega_p (0: omega_p = omega)
    int scalar;           // 1: a passive scalar T is stored after the flow fields (Eq. ACM2.0t)
    float at;             // 1 - 6 alpha = 2(omega_t - 1)/omega_t of the scalar
    int bulk;             // 1: D2Q9 bulk-viscosity variant, the trace Tr+ stored after the flow fields
    float gamma;          // its gamma (Appendix "Computing derivatives locally")
    int walled[3];      // 1 = half-way walls on both ends of this axis
    int lid_axis;       // axis whose top wall moves with the lid velocity
    int xfaces_done;    // 1: the interior kernel applied the x-face walls (inner x-face nodes)
    unsigned *sr_ctr;   // non-null: round stores stochastically, keyed by this step counter
    float *nup_p;       // omega_p on the half-row kernel: scratch for sum_i w_i c_i . J(x - c_i)
    int *err;           // device error word (bounded waits that gave up set it)
};

// The post-combine momentum a rho(x) u(x) of Eq. ACM2.0b(c), added to the partial
// sum j of the streamed link values: with rho = 1 + d and a = 1 + am1 (am1 = -6 nu),
// a rho u = u + m u where m = a d + am1 = post_factor(a, d, am1), so that
//     j + a rho u = (j + m u) + u.
// a rho itself is O(1): rounded to FP32, its error (up to 2^-24) depends only on the
// low bits of d, which move by a small fraction of an ulp per step, so the error
// keeps its sign at a node over hundreds of steps and the velocity drifts linearly
// (6e-5 u0 after 1000 steps of the 3D Taylor-Green workload against 4e-6 in this
// form). Here every rounded quantity is either small (m) or velocity-sized, and a
// velocity's low bits change every step.
__device__ __forceinline__ float post_factor(float a, float d, float am1) { return fmaf(a, d, am1); }
__device__ __forceinline__ float post_combine(float j, float m, float u) { return fmaf(m, u, j) + u; }

// g_i at a node with fields (d, u), for a link with integer velocity (cx,cy,cz)
// and weight w; q = |u|^2.
__device__ __forceinline__ float link_g(float w, float d, float rho, float e, float q, float s) {
    return w * (d + rho * fmaf(e, fmaf(4.5f, e, s), -1.5f * q));
}

}  // namespace lwacm
