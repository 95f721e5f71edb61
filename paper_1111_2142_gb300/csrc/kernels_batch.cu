// Batched update of many independent periodic domains of different sizes and
// viscosities, packed one after the other in the same field arrays.
//
// The domains are cut into tiles of 256 consecutive nodes (a tile never spans two
// domains); a CTA walks the tile list with a grid stride, one node per thread,
// and updates it with the per-node moment form of Eq. ACM2.0 (node_update.cuh)
// using its domain's (nx, ny, nz, nu).
//
//   k_batch_step        one launch = one step of every domain (the host replays
//                       the steps from captured CUDA graphs);
//   k_batch_persistent  one cooperative launch runs all the steps: the CTAs meet
//                       at a grid-wide barrier between steps. The barrier spins a
//                       bounded number of times; a CTA that gives up sets the
//                       device error word to 2 and returns, so a missing arrival
//                       ends the launch instead of hanging it.
//
// D2Q9 domains can instead be cut into 2D tiles of TW x TH nodes (shape chosen per
// context, by option or by the autotuner). A CTA of (TW+2) x (TH+2) threads takes
// one tile plus a one-node frame: every thread loads its node, computes the
// node's eight moving link values once (pre-combining, Eq. ACM2.0b(a)) and leaves
// them in shared memory; after a barrier each interior thread gathers the eight
// values arriving from its neighbours (streaming, Eq. ACM2.0b(b)) and forms the new
// moments (post-combining, Eq. ACM2.0b(c)).
#include <cooperative_groups.h>

#include "dev_cache.h"
#include "launch.h"
#include "lwacm_core.cuh"
#include "node_update.cuh"

namespace lwacm {
namespace {

constexpr int kTile = 256;
constexpr int kBarrierPolls = 1 << 21;  // with 256 ns back-off: well under a second

template <int Q, typename T>
__device__ __forceinline__ void tile_update(const T *__restrict__ in, T *__restrict__ out,
                                            const BatchParams &bp, long long t) {
    const BatchTile tile = bp.tiles[t];
    const BatchDomain dm = bp.doms[tile.dom];
    const long long k = tile.start + threadIdx.x;
    if (k >= dm.off + dm.n) return;
    const long long local = k - dm.off;
    StepParams p;
    p.nx = dm.nx;
    p.ny = dm.ny;
    p.nz = dm.nz;
    p.bc = BC_PERIODIC;
    p.N = dm.n;
    p.fstride = bp.fstride;
    p.s = dm.s;
    p.a = dm.a;
    p.am1 = dm.s * (-1.f / 3.f);
    p.wallc = 0.f;
    p.has_force = 0;
    p.gfield = nullptr;
    p.sdelta = 0.f;
    p.scalar = 0;
    p.bulk = 0;
    p.gamma = 0.f;
    p.at = 0.f;
    p.lid_axis = 0;
    p.err = nullptr;
    for (int c = 0; c < 3; ++c) {
        p.lid[c] = 0.f;
        p.force[c] = 0.f;
        p.walled[c] = 0;
    }
    int x, y, z;
    if (dm.n <= 0x7fffffffLL) {  // 32-bit index arithmetic (a 64-bit division costs several times more)
        const unsigned i = (unsigned)local, nx = (unsigned)dm.nx, r = i / nx;
        x = (int)(i - r * nx);
        y = (int)(r % (unsigned)dm.ny);
        z = (int)(r / (unsigned)dm.ny);
    } else {
        x = (int)(local % dm.nx);
        const long long r = local / dm.nx;
        y = (int)(r % dm.ny);
        z = (int)(r / dm.ny);
    }
    node_update<Q, false>(in + dm.off, out + dm.off, p, x, y, z);
}

// ---- 2D tiles (D2Q9) -------------------------------------------------------------
// link order of Lat<9>: 1 (1,0) 2 (-1,0) 3 (0,1) 4 (0,-1) 5 (1,1) 6 (-1,-1) 7 (1,-1) 8 (-1,1)
constexpr int kShapes[][2] = {{0, 0}, {30, 6}, {30, 14}, {62, 6}, {30, 30}, {62, 14}, {126, 6}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// walls of a single D2Q9 domain for the tile kernel (half-way walls on the walled
// axes, Eqs. ACM2.0cccbb2 / ACM2.0ccccbb; the lid moves on the top of lid axis)
struct Walls2 {
    int wx, wy;        // 1 = walls on both ends of x / y
    int lid_axis;      // 0: x, 1: y
    float wallc;       // 36 nu rho0
    float lidx, lidy;  // lid velocity
};

// forcing of a single D2Q9 domain (Eq. force): rho(x,t) (g + g(x)) added to j, with a
// constant acceleration g and an optional per-node field g(x) (two FP32 fields)
struct Force2 {
    int on = 0;
    float gx = 0.f, gy = 0.f;
    const float *field = nullptr;
    long long fstride = 0;
};

// one TW x TH tile (plus frame) of a D2Q9 domain whose node (0,0) is at packed
// index base; s, a: 18 nu and 1 - 6 nu of the domain. Without WALLS every axis is
// periodic; with WALLS a link whose source lies beyond a walled face takes the
// node's own value of the opposite link plus the moving-wall term. With BULK
// (periodic) the source's equilibrium is the quasi-equilibrium f^(e*) of Appendix
// "Computing derivatives locally": each source adds to its eight link values the
// increment Df - a Df^o of its trace deviation (the fourth field, Tr^(+) - Tr^(e)),
// with h = gamma (Tr^(+) - Tr^(e)) / 2,
//   Df = rho [h (ax B + ay A) + ax ay h^2],  Df^o = rho h (ax c_y v + ay c_x u) / 2,
// A = 1 - Pxx (c_x = 0) or (Pxx + c_x u)/2, ax = -1 or 1/2 (B, ay likewise in y),
// Pxx = 1/3 + u^2, Pyy = 1/3 + v^2; the rest link's increment stays with the node;
// the node stores Tr^(+) - Tr^(e) = sum_i (|c_i|^2 - 2/3) g_i / (1 + d+) - |u+|^2.
// With NUP (periodic; omega_p of Section 2.2, item 3) the density sums its link
// values with s_p = s + sdelta: d+ gains sdelta sum_i w_i rho e_i over the upwind
// sources; each source leaves W_p = w_p rho (c_p.u) of its four pairs in O, and the
// node takes sum_p [W_p(x - c_p) - W_p(x + c_p)] (the -c link carries -W_p). With
// BULK as well the density also takes (sdelta / 3) sum_i Df^o_i over the upwind
// sources (it pre-combines the increment with a_p, the momentum and the trace keep
// a): Df^o = kappa (c.u) with kappa = -rho h / 2 (axis), rho h / 4 (diagonal), so
// W_p becomes (w_p rho + kappa_p / 3) (c_p.u); the trace is normalised by the
// zeroth moment of the distribution built with a (the density before the sdelta
// terms).
template <int TW, int TH, typename T, bool WALLS = false, bool BULK = false, bool NUP = false>
__device__ __forceinline__ void tile2_core(const T *__restrict__ in, T *__restrict__ out, long long base, int nx,
                                           int ny, long long fstride, float s, float a, int x0, int y0,
                                           float (*G)[(TW + 2) * (TH + 2)], const Walls2 &wl = Walls2{},
                                           const Force2 &fc = Force2{}, float gamma = 0.f,
                                           float (*O)[(TW + 2) * (TH + 2)] = nullptr, float sdelta = 0.f) {
    constexpr int W = TW + 2;
    const int tx = threadIdx.x % W, ty = threadIdx.x / W;
    // periodic wrap of the frame (x0 + tx - 1 lies in [-1, x0 + TW], below 2 nx
    // whenever nx > TW; smaller domains take the modulo)
    int x = x0 + tx - 1, y = y0 + ty - 1;
    if (nx > TW) {
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    } else {
        x %= nx;
        if (x < 0) x += nx;
    }
    if (ny > TH) {
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    } else {
        y %= ny;
        if (y < 0) y += ny;
    }
    const long long k = base + (long long)y * nx + x;
    const float d = ldf(in + k), u = ldf(in + fstride + k), v = ldf(in + 2 * fstride + k);
    const float rho = 1.f + d;
    const float K = fmaf(-1.5f * rho, fmaf(u, u, v * v), d);  // d - 3/2 rho |u|^2
    const float nu = s * (1.f / 18.f);
    float df0 = 0.f;  // BULK: the rest link's increment
    {
        // pair (c, -c) with e = c.u: w (K + 9/2 rho e^2) +- w rho s e
        const float a9 = rho * nu * 2.f, b9 = rho * 0.5f, k9 = K * (1.f / 9.f);        // axis, w = 1/9
        const float a36 = rho * nu * 0.5f, b36 = rho * 0.125f, k36 = K * (1.f / 36.f);  // diagonal, w = 1/36
        const float e[4] = {u, v, u + v, u - v};
        // BULK: Df - a Df^o of the pair (c, -c) is an even part plus an odd part
        // proportional to e = c.u; with P = Pxx + Pyy and T = rho h (1 - a) / 4
        //   axis:     rho h (1 - P - h) / 2  -+ 2 T e
        //   diagonal: rho h (h + P) / 4      +- T e
        //   rest:     rho h (h - 2 + P)
        // (they sum to 0 in mass and momentum and to 2 rho h in the trace)
        float cax = 0.f, cdg = 0.f, oax = 0.f, odg = 0.f, kax = 0.f, kdg = 0.f;
        if (BULK) {
            const float h = 0.5f * gamma * ldf(in + 3 * fstride + k), rh = rho * h;
            const float P = fmaf(u, u, fmaf(v, v, 2.f / 3.f));
            cax = 0.5f * rh * (1.f - P - h);
            cdg = 0.25f * rh * (h + P);
            odg = 0.25f * rh * (1.f - a);
            oax = -2.f * odg;
            df0 = rh * (h - 2.f + P);
            kax = -0.5f * rh;
            kdg = 0.25f * rh;
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const bool dg = p >= 2;
            float cm = fmaf((dg ? b36 : b9) * e[p], e[p], dg ? k36 : k9);
            float A = dg ? a36 : a9;
            if (BULK) {  // (no + 0.f in the plain kernel: it would not fold away)
                cm += dg ? cdg : cax;
                A += dg ? odg : oax;
            }
            G[2 * p][threadIdx.x] = fmaf(A, e[p], cm);
            G[2 * p + 1][threadIdx.x] = fmaf(-A, e[p], cm);
            if (NUP && !BULK) O[p][threadIdx.x] = (dg ? rho * (1.f / 36.f) : rho * (1.f / 9.f)) * e[p];
            if (NUP && BULK)
                O[p][threadIdx.x] = fmaf(1.f / 3.f, dg ? kdg : kax, dg ? rho * (1.f / 36.f) : rho * (1.f / 9.f)) * e[p];
        }
    }
    __syncthreads();
    const int xi = x0 + tx - 1, yi = y0 + ty - 1;
    if (tx >= 1 && tx <= TW && ty >= 1 && ty <= TH && xi < nx && yi < ny) {
        const int tid = (int)threadIdx.x;
        // G[] order: (1,0) (-1,0) (0,1) (0,-1) (1,1) (-1,-1) (1,-1) (-1,1); the value
        // arriving along c comes from the neighbour at (tx - cx, ty - cy)
#define LW_IN(i, cx, cy) G[(i) - 1][tid - (cx) - (cy) * W]
        float g1 = LW_IN(1, 1, 0), g2 = LW_IN(2, -1, 0), g3 = LW_IN(3, 0, 1), g4 = LW_IN(4, 0, -1);
        float g5 = LW_IN(5, 1, 1), g6 = LW_IN(6, -1, -1), g7 = LW_IN(7, 1, -1), g8 = LW_IN(8, -1, 1);
#undef LW_IN
        if (WALLS) {
            const bool xl = wl.wx && xi == 0, xh = wl.wx && xi == nx - 1;
            const bool yl = wl.wy && yi == 0, yh = wl.wy && yi == ny - 1;
            if (xl || xh || yl || yh) {
                // link i with c = (cx, cy) from outside: own value along -c, plus the
                // lid term when the source lies beyond the top of the lid axis
                auto fix = [&](float &g, int i, int cx, int cy) {
                    const bool ox = (cx > 0 && xl) || (cx < 0 && xh), oy = (cy > 0 && yl) || (cy < 0 && yh);
                    if (!(ox || oy)) return;
                    const int j = (i & 1) ? i + 1 : i - 1;  // opposite link (pairs 1-2, 3-4, 5-6, 7-8)
                    float v = G[j - 1][tid];
                    const bool above = wl.lid_axis == 0 ? (cx < 0 && xh) : (cy < 0 && yh);
                    if (above) v = fmaf((i <= 4 ? 1.f / 9.f : 1.f / 36.f) * wl.wallc, cx * wl.lidx + cy * wl.lidy, v);
                    g = v;
                };
                fix(g1, 1, 1, 0);
                fix(g2, 2, -1, 0);
                fix(g3, 3, 0, 1);
                fix(g4, 4, 0, -1);
                fix(g5, 5, 1, 1);
                fix(g6, 6, -1, -1);
                fix(g7, 7, 1, -1);
                fix(g8, 8, -1, 1);
            }
        }
        const float s8 = ((g1 + g2) + (g3 + g4)) + ((g5 + g6) + (g7 + g8));
        const float g0 = BULK ? fmaf(4.f / 9.f, K, df0) : 0.f;  // BULK: the rest link
        float dd = BULK ? g0 + s8 : fmaf(4.f / 9.f, K, s8);
        const float rna = 1.f + dd;  // BULK: the trace's normalisation
        if (NUP) {
            const float dsp = (O[0][tid - 1] - O[0][tid + 1]) + (O[1][tid - W] - O[1][tid + W]) +
                              ((O[2][tid - 1 - W] - O[2][tid + 1 + W]) + (O[3][tid - 1 + W] - O[3][tid + 1 - W]));
            dd = fmaf(sdelta, dsp, dd);
        }
        const float m = post_factor(a, d, s * (-1.f / 3.f));  // a rho u = u + m u (post_combine)
        float jx = post_combine((g1 - g2) + ((g5 - g6) + (g7 - g8)), m, u);
        float jy = post_combine((g3 - g4) + ((g5 - g6) - (g7 - g8)), m, v);
        if (fc.on) {  // Eq. force: the odd part of f^(e)(rho(x,t), g) adds rho g to j
            jx = fmaf(rho, fc.gx, jx);
            jy = fmaf(rho, fc.gy, jy);
            if (fc.field) {
                const long long kf = (long long)yi * nx + xi;
                jx = fmaf(rho, __ldg(fc.field + kf), jx);
                jy = fmaf(rho, __ldg(fc.field + fc.fstride + kf), jy);
            }
        }
        const float rn = 1.f + dd;
        const float uxn = jx / rn, uyn = jy / rn;
        stf(out + k, dd);
        stf(out + fstride + k, uxn);
        stf(out + 2 * fstride + k, uyn);
        if (BULK) {  // |c|^2 - 2/3: rest -2/3, axis 1/3, diagonal 4/3
            const float trs = fmaf(-2.f / 3.f, g0,
                                   fmaf(1.f / 3.f, (g1 + g2) + (g3 + g4), (4.f / 3.f) * ((g5 + g6) + (g7 + g8))));
            stf(out + 3 * fstride + k, trs / rna - fmaf(uxn, uxn, uyn * uyn));
        }
    }
    __syncthreads();  // G is rewritten by the next tile
}

template <int TW, int TH, typename T>
__device__ __forceinline__ void tile2_update(const T *__restrict__ in, T *__restrict__ out, const BatchParams &bp,
                                             long long t, float (*G)[(TW + 2) * (TH + 2)]) {
    const BatchTile2 tile = bp.tiles2[t];
    const BatchDomain dm = bp.doms[tile.dom];
    tile2_core<TW, TH, T>(in, out, dm.off, dm.nx, dm.ny, bp.fstride, dm.s, dm.a, tile.x0, tile.y0, G);
}

// one D2Q9 domain, walls included (no separate wall pass); tiles numbered row-major
template <int TW, int TH, typename T, bool WALLS, bool BULK, bool NUP>
__global__ void __launch_bounds__((TW + 2) * (TH + 2)) k_d2q9_tiles(const T *__restrict__ in, T *__restrict__ out,
                                                                   int nx, int ny, long long fstride, float s,
                                                                   float a, int tilesx, long long ntiles, Walls2 wl,
                                                                   Force2 fc, float gamma, float sdelta) {
    __shared__ float G[8][(TW + 2) * (TH + 2)];
    __shared__ float O[NUP ? 4 : 1][(TW + 2) * (TH + 2)];
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const unsigned tu = (unsigned)t, ty = tu / (unsigned)tilesx;  // fewer than 2^32 tiles
        tile2_core<TW, TH, T, WALLS, BULK, NUP>(in, out, 0, nx, ny, fstride, s, a,
                                                (int)(tu - ty * (unsigned)tilesx) * TW, (int)ty * TH, G, wl, fc,
                                                gamma, O, sdelta);
    }
}

template <int TW, int TH, typename T>
__global__ void __launch_bounds__((TW + 2) * (TH + 2)) k_batch_tiles(const T *__restrict__ in, T *__restrict__ out,
                                                                    BatchParams bp) {
    __shared__ float G[8][(TW + 2) * (TH + 2)];
    for (long long t = blockIdx.x; t < bp.ntiles; t += gridDim.x) tile2_update<TW, TH, T>(in, out, bp, t, G);
}

template <int Q, typename T>
__global__ void __launch_bounds__(kTile) k_batch_step(const T *__restrict__ in, T *__restrict__ out,
                                                      BatchParams bp) {
    for (long long t = blockIdx.x; t < bp.ntiles; t += gridDim.x) tile_update<Q, T>(in, out, bp, t);
}

// Grid-wide barrier number `gen` (1, 2, ...): arrive on a counter, the last CTA
// resets it and publishes the generation; the others poll it, bounded.
__device__ bool grid_barrier(const BatchParams &bp, unsigned gen) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned arrived = atomicAdd(bp.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bp.bar_count, 0u);
            __threadfence();
            atomicExch(bp.bar_gen, gen);
        } else {
            ok = 0;
            for (int it = 0; it < kBarrierPolls; ++it) {
                if (atomicAdd(bp.bar_gen, 0u) >= gen) {
                    ok = 1;
                    break;
                }
                __nanosleep(256);
            }
            if (!ok) atomicExch(bp.err, 2);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <int Q, typename T>
__global__ void __launch_bounds__(kTile) k_batch_persistent(T *buf0, T *buf1, BatchParams bp,
                                                            long long nsteps, int parity) {
    for (long long s = 0; s < nsteps; ++s) {
        const int cur = (int)((parity + s) & 1);
        const T *in = cur ? buf1 : buf0;
        T *out = cur ? buf0 : buf1;
        for (long long t = blockIdx.x; t < bp.ntiles; t += gridDim.x) tile_update<Q, T>(in, out, bp, t);
        if (s + 1 < nsteps) {
            // test hook: CTA 0 leaves without arriving, so the others' waits run out
            if (bp.withhold_step == s && blockIdx.x == 0) return;
            if (!grid_barrier(bp, (unsigned)(s + 1))) return;
        }
    }
}

template <int TW, int TH, typename T>
__global__ void __launch_bounds__((TW + 2) * (TH + 2)) k_batch_tiles_persistent(T *buf0, T *buf1, BatchParams bp,
                                                                               long long nsteps, int parity) {
    __shared__ float G[8][(TW + 2) * (TH + 2)];
    for (long long s = 0; s < nsteps; ++s) {
        const int cur = (int)((parity + s) & 1);
        const T *in = cur ? buf1 : buf0;
        T *out = cur ? buf0 : buf1;
        for (long long t = blockIdx.x; t < bp.ntiles; t += gridDim.x) tile2_update<TW, TH, T>(in, out, bp, t, G);
        if (s + 1 < nsteps) {
            if (bp.withhold_step == s && blockIdx.x == 0) return;
            if (!grid_barrier(bp, (unsigned)(s + 1))) return;
        }
    }
}

// occupancy-limited grid of a kernel: CTAs per SM x SMs, cached per kernel and
// device (-1 when it cannot be determined)
template <typename K>
static int max_grid(K kern, int threads, DevSlots &cache) {
    return per_device(cache, [&] {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0) != cudaSuccess || per < 1)
            return -1;
        return per * device_sms();
    });
}

template <int TW, int TH, typename T>
cudaError_t tiles_t(const void *in, void *out, void *b0, void *b1, const BatchParams &bp, long long nsteps,
                    int parity, bool persistent, cudaStream_t st) {
    constexpr int NT = (TW + 2) * (TH + 2);
    if (!persistent) {
        static DevSlots cap;
        const int g = max_grid(k_batch_tiles<TW, TH, T>, NT, cap);
        if (g < 1) return cudaErrorNotSupported;
        const long long grid = bp.ntiles < 4LL * g ? bp.ntiles : 4LL * g;
        k_batch_tiles<TW, TH, T><<<(unsigned)grid, NT, 0, st>>>((const T *)in, (T *)out, bp);
        return cudaGetLastError();
    }
    static DevSlots cap;
    const int g = max_grid(k_batch_tiles_persistent<TW, TH, T>, NT, cap);
    if (g < 1) return cudaErrorNotSupported;
    const long long grid = bp.ntiles < g ? bp.ntiles : g;
    T *p0 = (T *)b0, *p1 = (T *)b1;
    BatchParams q = bp;
    void *args[] = {&p0, &p1, &q, &nsteps, &parity};
    return cudaLaunchCooperativeKernel((const void *)k_batch_tiles_persistent<TW, TH, T>, dim3((unsigned)grid),
                                       dim3(NT), args, 0, st);
}

template <typename T>
cudaError_t tiles_dispatch(const void *in, void *out, void *b0, void *b1, const BatchParams &bp, long long nsteps,
                           int parity, bool persistent, cudaStream_t st) {
    switch (bp.shape) {
        case 1: return tiles_t<30, 6, T>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
        case 2: return tiles_t<30, 14, T>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
        case 3: return tiles_t<62, 6, T>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
        case 4: return tiles_t<30, 30, T>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
        case 5: return tiles_t<62, 14, T>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
        case 6: return tiles_t<126, 6, T>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t tiles_storage(int storage, const void *in, void *out, void *b0, void *b1, const BatchParams &bp,
                          long long nsteps, int parity, bool persistent, cudaStream_t st) {
    switch (storage) {
        case STORE_F32: return tiles_dispatch<float>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
        case STORE_BF16: return tiles_dispatch<__nv_bfloat16>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
        case STORE_F16: return tiles_dispatch<__half>(in, out, b0, b1, bp, nsteps, parity, persistent, st);
    }
    return cudaErrorInvalidValue;
}

template <int TW, int TH, typename T, bool WALLS, bool BULK = false, bool NUP = false>
cudaError_t single_w(const void *in, void *out, const StepParams &p, const Walls2 &wl, cudaStream_t st) {
    constexpr int NT = (TW + 2) * (TH + 2);
    static DevSlots cap;
    const int g = max_grid(k_d2q9_tiles<TW, TH, T, WALLS, BULK, NUP>, NT, cap);
    if (g < 1) return cudaErrorNotSupported;
    const int tilesx = (p.nx + TW - 1) / TW;
    const long long ntiles = (long long)tilesx * ((p.ny + TH - 1) / TH);
    const long long grid = ntiles < 4LL * g ? ntiles : 4LL * g;
    Force2 fc;
    fc.on = p.has_force || p.gfield;
    fc.gx = p.has_force ? p.force[0] : 0.f;
    fc.gy = p.has_force ? p.force[1] : 0.f;
    fc.field = p.gfield;
    fc.fstride = p.fstride;
    k_d2q9_tiles<TW, TH, T, WALLS, BULK, NUP><<<(unsigned)grid, NT, 0, st>>>(
        (const T *)in, (T *)out, p.nx, p.ny, p.fstride, p.s, p.a, tilesx, ntiles, wl, fc, p.gamma, p.sdelta);
    return cudaGetLastError();
}

template <int TW, int TH, typename T>
cudaError_t single_t(const void *in, void *out, const StepParams &p, cudaStream_t st) {
    if (p.bulk && p.sdelta != 0.f) return single_w<TW, TH, T, false, true, true>(in, out, p, Walls2{}, st);
    if (p.bulk) return single_w<TW, TH, T, false, true>(in, out, p, Walls2{}, st);         // periodic only
    if (p.sdelta != 0.f) return single_w<TW, TH, T, false, false, true>(in, out, p, Walls2{}, st);  // periodic
    if (p.bc == BC_PERIODIC) return single_w<TW, TH, T, false>(in, out, p, Walls2{}, st);
    Walls2 wl;
    wl.wx = p.walled[0];
    wl.wy = p.walled[1];
    wl.lid_axis = p.lid_axis;
    wl.wallc = p.wallc;
    wl.lidx = p.lid[0];
    wl.lidy = p.lid[1];
    return single_w<TW, TH, T, true>(in, out, p, wl, st);
}

template <typename T>
cudaError_t single_dispatch(int shape, const void *in, void *out, const StepParams &p, cudaStream_t st) {
    switch (shape) {
        case 1: return single_t<30, 6, T>(in, out, p, st);
        case 2: return single_t<30, 14, T>(in, out, p, st);
        case 3: return single_t<62, 6, T>(in, out, p, st);
        case 4: return single_t<30, 30, T>(in, out, p, st);
        case 5: return single_t<62, 14, T>(in, out, p, st);
        case 6: return single_t<126, 6, T>(in, out, p, st);
    }
    return cudaErrorInvalidValue;
}

template <int Q, typename T>
cudaError_t persistent_t(void *b0, void *b1, const BatchParams &bp, long long nsteps, int parity,
                         cudaStream_t st) {
    static DevSlots cap;
    const int max_ctas = max_grid(k_batch_persistent<Q, T>, kTile, cap);
    if (max_ctas < 1) return cudaErrorNotSupported;
    const long long grid = bp.ntiles < max_ctas ? bp.ntiles : max_ctas;
    T *p0 = (T *)b0, *p1 = (T *)b1;
    BatchParams q = bp;
    void *args[] = {&p0, &p1, &q, &nsteps, &parity};
    return cudaLaunchCooperativeKernel((const void *)k_batch_persistent<Q, T>, dim3((unsigned)grid), dim3(kTile),
                                       args, 0, st);
}

template <typename T>
cudaError_t step_t(int Q, const void *in, void *out, const BatchParams &bp, cudaStream_t st) {
    const long long cap = (long long)device_sms() * 8;
    const unsigned grid = (unsigned)(bp.ntiles < cap ? bp.ntiles : cap);
    if (Q == 9)
        k_batch_step<9, T><<<grid, kTile, 0, st>>>((const T *)in, (T *)out, bp);
    else
        k_batch_step<19, T><<<grid, kTile, 0, st>>>((const T *)in, (T *)out, bp);
    return cudaGetLastError();
}

}  // namespace

int batch_tile() { return kTile; }
int batch_shapes() { return kNumShapes; }
void batch_shape(int k, int *tw, int *th) {
    const int i = k >= 0 && k < kNumShapes ? k : 0;
    *tw = kShapes[i][0];
    *th = kShapes[i][1];
}
bool batch_shape_supported(int Q, int storage, int k) {
    if (k == 0) return true;
    return Q == 9 && k > 0 && k < kNumShapes &&
           (storage == STORE_F32 || storage == STORE_BF16 || storage == STORE_F16);
}

bool tiles2d_supported(int Q, int storage, const StepParams &p) {
    // omega_p and the bulk variant (alone or together): periodic domains
    const bool variant_ok = (p.sdelta == 0.f && !p.bulk) || p.bc == BC_PERIODIC;
    return Q == 9 && p.nz == 1 && variant_ok && !p.scalar &&
           (storage == STORE_F32 || storage == STORE_BF16 || storage == STORE_F16);
}

cudaError_t launch_step_tiles2d(int Q, int storage, int shape, const void *in, void *out, const StepParams &p,
                                cudaStream_t st) {
    if (!tiles2d_supported(Q, storage, p) || shape < 1 || shape >= kNumShapes) return cudaErrorInvalidValue;
    switch (storage) {
        case STORE_F32: return single_dispatch<float>(shape, in, out, p, st);
        case STORE_BF16: return single_dispatch<__nv_bfloat16>(shape, in, out, p, st);
        case STORE_F16: return single_dispatch<__half>(shape, in, out, p, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_step(int Q, int storage, const void *in, void *out, const BatchParams &bp,
                              cudaStream_t st) {
    if (bp.shape > 0) {
        if (!batch_shape_supported(Q, storage, bp.shape)) return cudaErrorInvalidValue;
        return tiles_storage(storage, in, out, nullptr, nullptr, bp, 1, 0, false, st);
    }
    switch (storage) {
        case STORE_F32: return step_t<float>(Q, in, out, bp, st);
        case STORE_BF16: return step_t<__nv_bfloat16>(Q, in, out, bp, st);
        case STORE_F16: return step_t<__half>(Q, in, out, bp, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_persistent(int Q, int storage, void *buf0, void *buf1, const BatchParams &bp,
                                    long long nsteps, int parity, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bp.bar_count, 0, 2 * sizeof(unsigned), st);  // count, generation
    if (e != cudaSuccess) return e;
    if (bp.shape > 0) {
        if (!batch_shape_supported(Q, storage, bp.shape)) return cudaErrorInvalidValue;
        return tiles_storage(storage, nullptr, nullptr, buf0, buf1, bp, nsteps, parity, true, st);
    }
    if (Q == 9) {
        switch (storage) {
            case STORE_F32: return persistent_t<9, float>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_BF16: return persistent_t<9, __nv_bfloat16>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_F16: return persistent_t<9, __half>(buf0, buf1, bp, nsteps, parity, st);
        }
    } else {
        switch (storage) {
            case STORE_F32: return persistent_t<19, float>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_BF16: return persistent_t<19, __nv_bfloat16>(buf0, buf1, bp, nsteps, parity, st);
            case STORE_F16: return persistent_t<19, __half>(buf0, buf1, bp, nsteps, parity, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lwacm
