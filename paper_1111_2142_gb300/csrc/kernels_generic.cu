// Generic LW-ACM kernels: one thread per node, gathering (d,u) of the Q upwind
// neighbours through the cache hierarchy. Correct for every lattice, size,
// storage type and boundary type; the tiled kernels replace the interior update
// for the shapes they support. Also: the link-wise wall pass, field conversion
// and the FP64 diagnostics reduction.
#include <type_traits>

#include "launch.h"
#include "lwacm_core.cuh"
#include "node_update.cuh"
#include "tile_common.cuh"

namespace lwacm {

// Blocks of 32 x 8 nodes in an x-y plane when plane_blocks(p) (blockIdx = (x tile,
// y tile, z)), so that the y-neighbours of a block are mostly its own rows; else
// runs of 256 consecutive nodes.
__host__ __device__ inline bool plane_blocks(const StepParams &p) {
    return p.nx >= 32 && p.ny <= 8 * 65535 && p.nz <= 65535;
}
template <int Q, typename T, bool NUP, bool SC, bool BULK = false>
__global__ void __launch_bounds__(256) k_step_generic(const T *__restrict__ in,
                                                      T *__restrict__ out, StepParams p) {
    int x, y, z;
    if (plane_blocks(p)) {
        constexpr int BY = 8, BZ = 1;  // 32 x BY x BZ nodes per block (32 x 4 x 2 measured no faster in 3D)
        x = (int)(blockIdx.x * 32 + (threadIdx.x & 31));
        y = (int)(blockIdx.y * BY + ((threadIdx.x >> 5) % BY));
        z = (int)(blockIdx.z * BZ + (threadIdx.x >> 5) / BY);
        if (z >= p.nz) return;
        if (x >= p.nx || y >= p.ny) return;
        node_update<Q, false, NUP, SC, BULK>(in, out, p, x, y, z);
        return;
    }
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= p.N) return;
    if (p.N <= 0x7fffffffLL) {  // 32-bit index arithmetic (a 64-bit division costs several times more)
        const unsigned i = (unsigned)idx, nx = (unsigned)p.nx, r = i / nx;
        x = (int)(i - r * nx);
        y = (int)(r % (unsigned)p.ny);
        z = (int)(r / (unsigned)p.ny);
    } else {
        x = (int)(idx % p.nx);
        const long long r = idx / p.nx;
        y = (int)(r % p.ny);
        z = (int)(r / p.ny);
    }
    node_update<Q, false, NUP, SC, BULK>(in, out, p, x, y, z);
}

// Semi-implicit pressure update (Eq. FDcompact_si, Section 2.2 item 2), periodic
// domains: after the explicit step has written (d+, u+) to `out`, the density is
// summed again with every link value built from the old density (`in`) and the
// new velocity, d+(x) = sum_i g_i(d(x - c_i), u+(x - c_i)) with the link values of
// the moment form (lwacm_core.cuh; s_d = 18 nu, or 18 nu_p with omega_p). Reads
// the old density and the new velocity, writes only the new density.
template <int Q, typename T>
__global__ void __launch_bounds__(256) k_semi_implicit(const T *__restrict__ in, T *__restrict__ out,
                                                       StepParams p, float s_d) {
    using L = Lat<Q>;
    int x, y, z;
    if (plane_blocks(p)) {
        x = (int)(blockIdx.x * 32 + (threadIdx.x & 31));
        y = (int)(blockIdx.y * 8 + (threadIdx.x >> 5));
        z = (int)blockIdx.z;
        if (x >= p.nx || y >= p.ny || z >= p.nz) return;
    } else {
        const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (idx >= p.N) return;
        x = (int)(idx % p.nx);
        const long long r = idx / p.nx;
        y = (int)(r % p.ny);
        z = (int)(r / p.ny);
    }
    const T *Un = out + p.fstride, *Vn = out + 2 * p.fstride, *Wn = out + 3 * p.fstride;
    float dd = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        int sx = x - cx, sy = y - cy, sz = z - cz;
        sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
        sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
        sz = sz < 0 ? sz + p.nz : (sz >= p.nz ? sz - p.nz : sz);
        const long long s = ((long long)sz * p.ny + sy) * p.nx + sx;
        const float ds = ldf(in + s), us = ldf(Un + s), vs = ldf(Vn + s);
        const float ws = (Q == 19) ? ldf(Wn + s) : 0.f;
        const float e = cx * us + cy * vs + cz * ws;
        const float q = fmaf(us, us, fmaf(vs, vs, ws * ws));
        dd += link_g(L::w(i), ds, 1.f + ds, e, q, s_d);
    }
    stf(out + ((long long)z * p.ny + y) * p.nx + x, dd);
}

template <typename T>
cudaError_t launch_semi_implicit_t(int Q, const void *in, void *out, const StepParams &p, cudaStream_t st) {
    const dim3 nb = plane_blocks(p) ? dim3((unsigned)((p.nx + 31) / 32), (unsigned)((p.ny + 7) / 8), (unsigned)p.nz)
                                    : dim3((unsigned)((p.N + 255) / 256));
    const float s_d = p.s + p.sdelta;
    if (Q == 9)
        k_semi_implicit<9, T><<<nb, 256, 0, st>>>((const T *)in, (T *)out, p, s_d);
    else
        k_semi_implicit<19, T><<<nb, 256, 0, st>>>((const T *)in, (T *)out, p, s_d);
    return cudaGetLastError();
}

cudaError_t launch_semi_implicit(int Q, int storage, const void *in, void *out, const StepParams &p,
                                 cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return launch_semi_implicit_t<float>(Q, in, out, p, st);
        case STORE_BF16: return launch_semi_implicit_t<__nv_bfloat16>(Q, in, out, p, st);
        case STORE_F16: return launch_semi_implicit_t<__half>(Q, in, out, p, st);
    }
    return cudaErrorInvalidValue;
}

// Boundary nodes of a walled domain, enumerated without gaps.
//   cavity 2D: the perimeter of the nx x ny rectangle;
//   cavity 3D: the planes z = 0 and z = nz-1, then the perimeter of each inner plane;
//   channel:   rows y = 0 and y = ny-1 of every z plane.
__host__ __device__ inline long long perimeter(int nx, int ny) {
    return ny <= 1 ? nx : (nx <= 1 ? ny : 2LL * nx + 2LL * (ny - 2));
}
__host__ __device__ inline long long boundary_count(const StepParams &p, int D) {
    if (p.bc == BC_CHANNEL) return (p.ny <= 1 ? 1LL : 2LL) * p.nx * p.nz;
    if (D == 2) return perimeter(p.nx, p.ny);
    if (p.nz <= 2) return (long long)p.nx * p.ny * p.nz;
    return 2LL * p.nx * p.ny + (long long)(p.nz - 2) * perimeter(p.nx, p.ny);
}
__device__ inline void perimeter_node(long long t, int nx, int ny, int &x, int &y) {
    if (ny <= 1) { x = (int)t; y = 0; return; }
    if (nx <= 1) { x = 0; y = (int)t; return; }
    if (t < nx) { x = (int)t; y = 0; return; }
    t -= nx;
    if (t < nx) { x = (int)t; y = ny - 1; return; }
    t -= nx;
    if (t < ny - 2) { x = 0; y = 1 + (int)t; return; }
    t -= ny - 2;
    x = nx - 1;
    y = 1 + (int)t;
}

template <int Q, typename T>
__global__ void __launch_bounds__(256) k_wall_pass(const T *__restrict__ in, T *__restrict__ out,
                                                   StepParams p, long long nb) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    int x, y, z;
    if (p.bc == BC_CHANNEL) {
        const long long row = t / p.nx;  // 0 .. 2*nz-1
        x = (int)(t % p.nx);
        z = (int)(row >> 1);
        y = (row & 1) ? p.ny - 1 : 0;
    } else if (Q == 9 || p.nz <= 2) {
        if (Q == 9) {
            z = 0;
            perimeter_node(t, p.nx, p.ny, x, y);
        } else {  // every node is on the boundary
            x = (int)(t % p.nx);
            y = (int)((t / p.nx) % p.ny);
            z = (int)(t / ((long long)p.nx * p.ny));
        }
    } else {
        const long long plane = (long long)p.nx * p.ny;
        if (t < 2 * plane) {
            z = t < plane ? 0 : p.nz - 1;
            const long long r = t < plane ? t : t - plane;
            x = (int)(r % p.nx);
            y = (int)(r / p.nx);
        } else {
            const long long per = perimeter(p.nx, p.ny);
            const long long r = t - 2 * plane;
            z = 1 + (int)(r / per);
            perimeter_node(r % per, p.nx, p.ny, x, y);
        }
    }
    node_update<Q, true>(in, out, p, x, y, z);
}

// node_update<19, true> for a node of a cavity (every axis walled, so no source
// wraps): the wall test of each link reduces to the node's face flags and the
// source offsets to per-direction constants; same link order and arithmetic.
// I32: every element offset of the four fields fits 32-bit arithmetic (the caller
// checks 4 fstride < 2^31); the per-direction offsets are then formed once.
template <typename T, bool I32 = false>
__device__ __forceinline__ void cavity_node_update(const T *__restrict__ in, T *__restrict__ out,
                                                   const StepParams &p, int x, int y, int z) {
    using L = Lat<19>;
    using Idx = typename std::conditional<I32, int, long long>::type;
    const Idx plane = (Idx)p.nx * p.ny, nxi = (Idx)p.nx;
    const Idx k = (Idx)z * plane + (Idx)y * p.nx + x;
    const T *Din = in + k, *Uin = in + p.fstride + k, *Vin = in + 2 * p.fstride + k, *Win = in + 3 * p.fstride + k;
    const bool lo0 = x == 0, lo1 = y == 0, lo2 = z == 0;
    const bool hi0 = x == p.nx - 1, hi1 = y == p.ny - 1, hi2 = z == p.nz - 1;
    const int la = p.lid_axis;
    const float dx = ldf(Din), ux = ldf(Uin), uy = ldf(Vin), uz = ldf(Win);
    const float rx = 1.f + dx;
    const float qx = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    float dd = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        // the source x - c lies beyond the low face when c = +1, the high face when -1
        const bool bx = (cx > 0 && lo0) || (cx < 0 && hi0);
        const bool by = (cy > 0 && lo1) || (cy < 0 && hi1);
        const bool bz = (cz > 0 && lo2) || (cz < 0 && hi2);
        const bool outside = bx || by || bz;
        const bool above = (la == 0 ? cx < 0 && hi0 : (la == 1 ? cy < 0 && hi1 : cz < 0 && hi2));
        // a source beyond a wall reads the node itself (loaded already, unused)
        const Idx so = outside ? 0 : (Idx)cz * plane + (Idx)cy * nxi + cx;
        const float ds = ldf(Din - so), us = ldf(Uin - so), vs = ldf(Vin - so), ws = ldf(Win - so);
        float g;
        if (!outside) {
            const float e = cx * us + cy * vs + cz * ws;
            const float q = fmaf(us, us, fmaf(vs, vs, ws * ws));
            g = link_g(L::w(i), ds, 1.f + ds, e, q, p.s);
        } else {
            // Eq. ACM2.0cccbb2 + Eq. ACM2.0ccccbb: own outgoing BB(i) value, reflected
            const float e = -(cx * ux + cy * uy + cz * uz);
            g = link_g(L::w(i), dx, rx, e, qx, p.s);
            if (above) {
                const float cu = cx * p.lid[0] + cy * p.lid[1] + cz * p.lid[2];
                g = fmaf(L::w(i) * p.wallc, cu, g);
            }
        }
        dd += g;
        if (cx) jx += cx > 0 ? g : -g;
        if (cy) jy += cy > 0 ? g : -g;
        if (cz) jz += cz > 0 ? g : -g;
    }
    const float mx = post_factor(p.a, dx, p.am1);  // a rho u = u + mx u (post_combine)
    jx = post_combine(jx, mx, ux);
    jy = post_combine(jy, mx, uy);
    jz = post_combine(jz, mx, uz);
    if (p.has_force) {  // Eq. force
        jx = fmaf(rx, p.force[0], jx);
        jy = fmaf(rx, p.force[1], jy);
        jz = fmaf(rx, p.force[2], jz);
    }
    if (p.gfield) {
        jx = fmaf(rx, __ldg(p.gfield + k), jx);
        jy = fmaf(rx, __ldg(p.gfield + p.fstride + k), jy);
        jz = fmaf(rx, __ldg(p.gfield + 2 * p.fstride + k), jz);
    }
    // u = j / (1 + d+), the IEEE quotient without the checked division's branch
    const tile::Div1 r = tile::div_prep(1.f + dd);
    stf(out + k, dd);
    stf(out + p.fstride + k, tile::div_apply(jx, r));
    stf(out + 2 * p.fstride + k, tile::div_apply(jy, r));
    stf(out + 3 * p.fstride + k, tile::div_apply(jz, r));
}

// The same update for a node of a boundary row whose y and z faces are known at
// compile time (YF, ZF: 0 none, 1 the low face, 2 the high face; 32-bit offsets):
// a link that leaves through one of them bounces with neither a load nor a test,
// and only the x-face links (the row's two end nodes) keep a test. Same link order
// and arithmetic as cavity_node_update, so the same results.
template <typename T, int YF, int ZF>
__device__ __forceinline__ void cavity_row_update(const T *__restrict__ in, T *__restrict__ out,
                                                  const StepParams &p, int x, int y, int z) {
    using L = Lat<19>;
    const int plane = p.nx * p.ny;
    const int k = z * plane + y * p.nx + x;
    const T *Din = in + k, *Uin = in + p.fstride + k, *Vin = in + 2 * p.fstride + k, *Win = in + 3 * p.fstride + k;
    const bool lo0 = x == 0, hi0 = x == p.nx - 1;
    const int la = p.lid_axis;
    const float dx = ldf(Din), ux = ldf(Uin), uy = ldf(Vin), uz = ldf(Win);
    const float rx = 1.f + dx;
    const float qx = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    float dd = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        const bool byz = (cy > 0 && YF == 1) || (cy < 0 && YF == 2) || (cz > 0 && ZF == 1) || (cz < 0 && ZF == 2);
        const bool bx = (cx > 0 && lo0) || (cx < 0 && hi0);
        const bool above = la == 0 ? (cx < 0 && hi0) : (la == 1 ? (cy < 0 && YF == 2) : (cz < 0 && ZF == 2));
        float g;
        bool own = byz;
        if (!byz) {
            const int so = bx ? 0 : cz * plane + cy * p.nx + cx;
            const float ds = ldf(Din - so), us = ldf(Uin - so), vs = ldf(Vin - so), ws = ldf(Win - so);
            const float e = cx * us + cy * vs + cz * ws;
            const float q = fmaf(us, us, fmaf(vs, vs, ws * ws));
            g = link_g(L::w(i), ds, 1.f + ds, e, q, p.s);
            own = bx;
        }
        if (own) {
            // Eq. ACM2.0cccbb2 + Eq. ACM2.0ccccbb: own outgoing BB(i) value, reflected
            const float e = -(cx * ux + cy * uy + cz * uz);
            g = link_g(L::w(i), dx, rx, e, qx, p.s);
            if (above) {
                const float cu = cx * p.lid[0] + cy * p.lid[1] + cz * p.lid[2];
                g = fmaf(L::w(i) * p.wallc, cu, g);
            }
        }
        dd += g;
        if (cx) jx += cx > 0 ? g : -g;
        if (cy) jy += cy > 0 ? g : -g;
        if (cz) jz += cz > 0 ? g : -g;
    }
    const float mx = post_factor(p.a, dx, p.am1);  // a rho u = u + mx u (post_combine)
    jx = post_combine(jx, mx, ux);
    jy = post_combine(jy, mx, uy);
    jz = post_combine(jz, mx, uz);
    if (p.has_force) {  // Eq. force
        jx = fmaf(rx, p.force[0], jx);
        jy = fmaf(rx, p.force[1], jy);
        jz = fmaf(rx, p.force[2], jz);
    }
    if (p.gfield) {
        jx = fmaf(rx, __ldg(p.gfield + k), jx);
        jy = fmaf(rx, __ldg(p.gfield + p.fstride + k), jy);
        jz = fmaf(rx, __ldg(p.gfield + 2 * p.fstride + k), jz);
    }
    const tile::Div1 r = tile::div_prep(1.f + dd);
    stf(out + k, dd);
    stf(out + p.fstride + k, tile::div_apply(jx, r));
    stf(out + 2 * p.fstride + k, tile::div_apply(jy, r));
    stf(out + 3 * p.fstride + k, tile::div_apply(jz, r));
}

// D3Q19 cavity walls in one launch (k_wall_cavity3d) when the x faces have inner
// nodes (y in [1, ny-2], z in [1, nz-2]) with an inner column beside each (nx >= 2):
// blocks of shared-memory staged x-face patches, then blocks of boundary rows.
__host__ __device__ inline bool xface_split(const StepParams &p, int D) {
    return D == 3 && p.bc == BC_CAVITY && p.nx >= 2 && p.ny > 2 && p.nz > 2;
}
constexpr int WC_THREADS = 256;

// Boundary row r other than the inner x-face nodes (the ny rows of z = 0, those of
// z = nz-1, then y = 0 and y = ny-1 of each inner plane), node x of it: coalesced
// across a block, the row found once per block in 32-bit arithmetic.
__host__ __device__ inline long long wall_rows(const StepParams &p) { return 2LL * p.ny + 2LL * (p.nz - 2); }
template <typename T>
__device__ __forceinline__ void wall_row_node(const T *__restrict__ in, T *__restrict__ out, const StepParams &p,
                                              int r, int x) {
    int y, z;
    if (r < 2 * p.ny) {
        z = r < p.ny ? 0 : p.nz - 1;
        y = r < p.ny ? r : r - p.ny;
    } else {
        const int q = r - 2 * p.ny;
        z = 1 + (q >> 1);
        y = (q & 1) ? p.ny - 1 : 0;
    }
    if (4 * p.fstride >= 0x7fffffffLL) {
        cavity_node_update<T, false>(in, out, p, x, y, z);
        return;
    }
    const int yf = y == 0 ? 1 : (y == p.ny - 1 ? 2 : 0), zf = z == 0 ? 1 : (z == p.nz - 1 ? 2 : 0);
    switch (yf * 3 + zf) {  // uniform per block: one row
        case 1: cavity_row_update<T, 0, 1>(in, out, p, x, y, z); break;
        case 2: cavity_row_update<T, 0, 2>(in, out, p, x, y, z); break;
        case 3: cavity_row_update<T, 1, 0>(in, out, p, x, y, z); break;
        case 4: cavity_row_update<T, 1, 1>(in, out, p, x, y, z); break;
        case 5: cavity_row_update<T, 1, 2>(in, out, p, x, y, z); break;
        case 6: cavity_row_update<T, 2, 0>(in, out, p, x, y, z); break;
        case 7: cavity_row_update<T, 2, 1>(in, out, p, x, y, z); break;
        case 8: cavity_row_update<T, 2, 2>(in, out, p, x, y, z); break;
        default: cavity_node_update<T, true>(in, out, p, x, y, z); break;
    }
}

// The inner nodes of the x = 0 and x = nx-1 faces of a D3Q19 cavity (patch (py, pz)
// of face `face`; y in [1, ny-2], z in [1, nz-2]): one thread per node, but
// their sources (own and inner column, y and z within one) are first staged in
// shared memory for a patch of XF_PY x XF_PZ nodes. With x fastest in memory, one
// thread per face node gathering straight from global memory sends every warp load
// to 32 rows (32 sectors) and overflows L1 with lines of which 8 bytes are used;
// here each needed row sector is requested once per patch. The update is
// node_update<19, true> restated for these nodes (same link order and arithmetic,
// so the same results): only x-links can leave the box, the lid applies when it
// moves the x = nx-1 face.
constexpr int XF_PY = 32, XF_PZ = 8, XF_RY = XF_PY + 2, XF_RZ = XF_PZ + 2;
static_assert(XF_PY * XF_PZ == WC_THREADS, "one thread per patch node");
template <typename T>
__device__ __forceinline__ void xface_patch(const T *__restrict__ in, T *__restrict__ out, const StepParams &p,
                                            int face, int py, int pz) {
    using L = Lat<19>;
    __shared__ float sm[4][XF_RZ][XF_RY][2];  // [field][z][y][own column, inner column]
    const int xo = face ? p.nx - 1 : 0, xi = face ? p.nx - 2 : 1;
    const int y0 = 1 + py * XF_PY, z0 = 1 + pz * XF_PZ;
    // every load of the patch issued before the first shared store (NL per thread)
    constexpr int NR = XF_RY * XF_RZ, NE = 4 * NR * 2, NT = WC_THREADS, NL = (NE + NT - 1) / NT;
    float v[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        const int e = (int)threadIdx.x + j * NT;
        const int col = e & 1, r = (e >> 1) % NR, f = (e >> 1) / NR;
        const int y = y0 - 1 + r % XF_RY, z = z0 - 1 + r / XF_RY;  // >= 0: y0, z0 >= 1
        v[j] = 0.f;
        if (e < NE && y < p.ny && z < p.nz)
            v[j] = ldf(in + (long long)f * p.fstride + ((long long)z * p.ny + y) * p.nx + (col ? xi : xo));
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        const int e = (int)threadIdx.x + j * NT;
        if (e < NE) (&sm[0][0][0][0])[e] = v[j];  // [f][z][y][col] is e's own order
    }
    __syncthreads();
    const int ty = (int)threadIdx.x % XF_PY, tz = (int)threadIdx.x / XF_PY;
    const int y = y0 + ty, z = z0 + tz;
    if (y > p.ny - 2 || z > p.nz - 2) return;
    const long long k = ((long long)z * p.ny + y) * p.nx + xo;
    const float dx = sm[0][tz + 1][ty + 1][0], ux = sm[1][tz + 1][ty + 1][0], uy = sm[2][tz + 1][ty + 1][0];
    const float uz = sm[3][tz + 1][ty + 1][0];
    const float rx = 1.f + dx;
    const float qx = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const bool lid_face = face == 1 && p.lid_axis == 0;
    float dd = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        const bool outside = cx == (face ? -1 : 1);  // source x - cx beyond the wall
        float g;
        if (!outside) {
            const int c = cx == 0 ? 0 : 1, yy = ty + 1 - cy, zz = tz + 1 - cz;
            const float ds = sm[0][zz][yy][c], us = sm[1][zz][yy][c], vs = sm[2][zz][yy][c];
            const float ws = sm[3][zz][yy][c];
            const float e = cx * us + cy * vs + cz * ws;
            const float q = fmaf(us, us, fmaf(vs, vs, ws * ws));
            g = link_g(L::w(i), ds, 1.f + ds, e, q, p.s);
        } else {
            // Eq. ACM2.0cccbb2 + Eq. ACM2.0ccccbb: own outgoing BB(i) value, reflected
            const float e = -(cx * ux + cy * uy + cz * uz);
            g = link_g(L::w(i), dx, rx, e, qx, p.s);
            if (lid_face) {
                const float cu = cx * p.lid[0] + cy * p.lid[1] + cz * p.lid[2];
                g = fmaf(L::w(i) * p.wallc, cu, g);
            }
        }
        dd += g;
        if (cx) jx += cx > 0 ? g : -g;
        if (cy) jy += cy > 0 ? g : -g;
        if (cz) jz += cz > 0 ? g : -g;
    }
    const float mx = post_factor(p.a, dx, p.am1);  // a rho u = u + mx u (post_combine)
    jx = post_combine(jx, mx, ux);
    jy = post_combine(jy, mx, uy);
    jz = post_combine(jz, mx, uz);
    if (p.has_force) {  // Eq. force
        jx = fmaf(rx, p.force[0], jx);
        jy = fmaf(rx, p.force[1], jy);
        jz = fmaf(rx, p.force[2], jz);
    }
    if (p.gfield) {
        jx = fmaf(rx, __ldg(p.gfield + k), jx);
        jy = fmaf(rx, __ldg(p.gfield + p.fstride + k), jy);
        jz = fmaf(rx, __ldg(p.gfield + 2 * p.fstride + k), jz);
    }
    const float rn = 1.f + dd;
    stf(out + k, dd);
    stf(out + p.fstride + k, jx / rn);
    stf(out + 2 * p.fstride + k, jy / rn);
    stf(out + 3 * p.fstride + k, jz / rn);
}

// blocks [0, 2 npy npz): x-face patches (face, py, pz), py fastest; then bpr blocks
// per boundary row
template <typename T>
__global__ void __launch_bounds__(WC_THREADS) k_wall_cavity3d(const T *__restrict__ in, T *__restrict__ out,
                                                              StepParams p, int npy, int npz, int bpr) {
    const int b = (int)blockIdx.x, nxf = 2 * npy * npz;
    if (b < nxf) {
        xface_patch(in, out, p, b / (npy * npz), b % npy, (b / npy) % npz);
        return;
    }
    const int rb = b - nxf, x = (rb % bpr) * WC_THREADS + (int)threadIdx.x;
    if (x < p.nx) wall_row_node(in, out, p, rb / bpr, x);
}

// storage -> double needs the exact stored value, converted without rounding
template <typename T>
__global__ void k_to_f64(const T *__restrict__ in, double *__restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)ldf(in + i);
}
template <typename T>
__global__ void k_to_f32(const T *__restrict__ in, float *__restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = ldf(in + i);
}
template <typename Ti, typename T>
__global__ void k_from(const Ti *__restrict__ in, T *__restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if constexpr (sizeof(Ti) == 8) {
            // round once from FP64 to the storage type
            if constexpr (sizeof(T) == 4)
                out[i] = __double2float_rn(in[i]);
            else if constexpr (std::is_same<T, __half>::value)
                out[i] = __double2half(in[i]);
            else
                out[i] = __double2bfloat16(in[i]);
        } else {
            stf(out + i, in[i]);
        }
    }
}

// ---- FP64 diagnostics: per-block partials, then one block in fixed order ------
constexpr int kDiagVals = 9;  // mass, jx, jy, jz, ke, max|u|^2, mpar, mperp, nonfinite

template <typename T>
__global__ void __launch_bounds__(256) k_diag_partial(const T *__restrict__ f, long long fstride,
                                                      long long N, int has_z,
                                                      double *__restrict__ partial) {
    double acc[kDiagVals] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = ldf(f + i), u = ldf(f + fstride + i), v = ldf(f + 2 * fstride + i);
        const double w = has_z ? (double)ldf(f + 3 * fstride + i) : 0.0;
        const double rho = 1.0 + d, uu = u * u + v * v + w * w;
        acc[0] += d;
        acc[1] += rho * u;
        acc[2] += rho * v;
        acc[3] += rho * w;
        acc[4] += 0.5 * rho * uu;
        acc[5] = fmax(acc[5], uu);
        if (has_z) {
            // Eq. 3Dmomenta, read for a lid moving along the x = y diagonal of the
            // top z plane: components parallel / perpendicular to the lid (times sqrt 2)
            acc[6] += 0.5 * (u + v) * (u + v);
            acc[7] += 0.5 * (u - v) * (u - v);
        }
        if (!isfinite(d) || !isfinite(uu)) acc[8] += 1.0;
    }
    __shared__ double sh[kDiagVals][256];
    for (int v = 0; v < kDiagVals; ++v) sh[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int v = 0; v < kDiagVals; ++v) {
                const double o = sh[v][threadIdx.x + off];
                sh[v][threadIdx.x] = (v == 5) ? fmax(sh[v][threadIdx.x], o) : sh[v][threadIdx.x] + o;
            }
        __syncthreads();
    }
    if (threadIdx.x < kDiagVals) partial[(long long)blockIdx.x * kDiagVals + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_diag_final(const double *__restrict__ partial, int nblocks, double *__restrict__ out) {
    __shared__ double sh[kDiagVals][256];
    double acc[kDiagVals] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int v = 0; v < kDiagVals; ++v) {
            const double o = partial[(long long)b * kDiagVals + v];
            acc[v] = (v == 5) ? fmax(acc[v], o) : acc[v] + o;
        }
    for (int v = 0; v < kDiagVals; ++v) sh[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int v = 0; v < kDiagVals; ++v) {
                const double o = sh[v][threadIdx.x + off];
                sh[v][threadIdx.x] = (v == 5) ? fmax(sh[v][threadIdx.x], o) : sh[v][threadIdx.x] + o;
            }
        __syncthreads();
    }
    if (threadIdx.x < kDiagVals) out[threadIdx.x] = sh[threadIdx.x][0];
}

// ---- host launchers ---------------------------------------------------------
static inline unsigned blocks_for(long long n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

template <typename T>
cudaError_t launch_step_generic_t(int Q, const void *in, void *out, const StepParams &p,
                                  cudaStream_t st) {
    const int by = 8, bz = 1;
    const dim3 nb = plane_blocks(p) ? dim3((unsigned)((p.nx + 31) / 32), (unsigned)((p.ny + by - 1) / by),
                                           (unsigned)((p.nz + bz - 1) / bz))
                                    : dim3(blocks_for(p.N, 256));
    const int v = (p.sdelta != 0.f ? 1 : 0) + (p.scalar ? 2 : 0) + (p.bulk ? 4 : 0);
    const T *i0 = (const T *)in;
    T *o0 = (T *)out;
    if (Q == 9) {
        switch (v) {
            case 0: k_step_generic<9, T, false, false><<<nb, 256, 0, st>>>(i0, o0, p); break;
            case 1: k_step_generic<9, T, true, false><<<nb, 256, 0, st>>>(i0, o0, p); break;
            case 2: k_step_generic<9, T, false, true><<<nb, 256, 0, st>>>(i0, o0, p); break;
            case 3: k_step_generic<9, T, true, true><<<nb, 256, 0, st>>>(i0, o0, p); break;
            case 4: k_step_generic<9, T, false, false, true><<<nb, 256, 0, st>>>(i0, o0, p); break;
            case 5: k_step_generic<9, T, true, false, true><<<nb, 256, 0, st>>>(i0, o0, p); break;
            default: return cudaErrorInvalidValue;  // the scalar and the trace share one field
        }
    } else {
        switch (v) {
            case 0: k_step_generic<19, T, false, false><<<nb, 256, 0, st>>>(i0, o0, p); break;
            case 1: k_step_generic<19, T, true, false><<<nb, 256, 0, st>>>(i0, o0, p); break;
            case 2: k_step_generic<19, T, false, true><<<nb, 256, 0, st>>>(i0, o0, p); break;
            default: k_step_generic<19, T, true, true><<<nb, 256, 0, st>>>(i0, o0, p); break;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_step_generic(int Q, int storage, const void *in, void *out,
                                const StepParams &p, cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return launch_step_generic_t<float>(Q, in, out, p, st);
        case STORE_BF16: return launch_step_generic_t<__nv_bfloat16>(Q, in, out, p, st);
        case STORE_F16: return launch_step_generic_t<__half>(Q, in, out, p, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_wall_t(int Q, const void *in, void *out, const StepParams &p, cudaStream_t st) {
    const long long nb = boundary_count(p, Q == 9 ? 2 : 3);
    if (nb <= 0) return cudaSuccess;
    if (Q == 19 && xface_split(p, 3)) {
        // the inner x-face nodes in staged patches, unless the interior kernel did them
        const long long npy = p.xfaces_done ? 0 : (p.ny - 2 + XF_PY - 1) / XF_PY;
        const long long npz = p.xfaces_done ? 0 : (p.nz - 2 + XF_PZ - 1) / XF_PZ;
        const long long bpr = (p.nx + WC_THREADS - 1) / WC_THREADS;
        const long long blocks = 2 * npy * npz + wall_rows(p) * bpr;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        k_wall_cavity3d<T><<<(unsigned)blocks, WC_THREADS, 0, st>>>((const T *)in, (T *)out, p, (int)npy, (int)npz,
                                                                    (int)bpr);
    } else if (Q == 9) {
        k_wall_pass<9, T><<<blocks_for(nb, 256), 256, 0, st>>>((const T *)in, (T *)out, p, nb);
    } else {
        k_wall_pass<19, T><<<blocks_for(nb, 256), 256, 0, st>>>((const T *)in, (T *)out, p, nb);
    }
    return cudaGetLastError();
}

cudaError_t launch_wall_pass(int Q, int storage, const void *in, void *out, const StepParams &p,
                             cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return launch_wall_t<float>(Q, in, out, p, st);
        case STORE_BF16: return launch_wall_t<__nv_bfloat16>(Q, in, out, p, st);
        case STORE_F16: return launch_wall_t<__half>(Q, in, out, p, st);
    }
    return cudaErrorInvalidValue;
}

static unsigned conv_blocks(long long n) {
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

template <typename T>
static cudaError_t from_t(int src_dtype, const void *src, void *dst, long long n, cudaStream_t st) {
    if (src_dtype == XFER_F64)
        k_from<double, T><<<conv_blocks(n), 256, 0, st>>>((const double *)src, (T *)dst, n);
    else
        k_from<float, T><<<conv_blocks(n), 256, 0, st>>>((const float *)src, (T *)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_in(int storage, int src_dtype, const void *src, void *dst, long long n,
                              cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return from_t<float>(src_dtype, src, dst, n, st);
        case STORE_BF16: return from_t<__nv_bfloat16>(src_dtype, src, dst, n, st);
        case STORE_F16: return from_t<__half>(src_dtype, src, dst, n, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t to_t(int dst_dtype, const void *src, void *dst, long long n, cudaStream_t st) {
    if (dst_dtype == XFER_F64)
        k_to_f64<T><<<conv_blocks(n), 256, 0, st>>>((const T *)src, (double *)dst, n);
    else
        k_to_f32<T><<<conv_blocks(n), 256, 0, st>>>((const T *)src, (float *)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_out(int storage, int dst_dtype, const void *src, void *dst, long long n,
                               cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return to_t<float>(dst_dtype, src, dst, n, st);
        case STORE_BF16: return to_t<__nv_bfloat16>(dst_dtype, src, dst, n, st);
        case STORE_F16: return to_t<__half>(dst_dtype, src, dst, n, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t diag_t(const void *f, long long fstride, long long N, int has_z, double *partial,
                          double *out, cudaStream_t st) {
    k_diag_partial<T><<<kDiagBlocks, 256, 0, st>>>((const T *)f, fstride, N, has_z, partial);
    k_diag_final<<<1, 256, 0, st>>>(partial, kDiagBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(int storage, const void *f, long long fstride, long long N,
                               int has_z, double *partial, double *out, cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return diag_t<float>(f, fstride, N, has_z, partial, out, st);
        case STORE_BF16: return diag_t<__nv_bfloat16>(f, fstride, N, has_z, partial, out, st);
        case STORE_F16: return diag_t<__half>(f, fstride, N, has_z, partial, out, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lwacm
