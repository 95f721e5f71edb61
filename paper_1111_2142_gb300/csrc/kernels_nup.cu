// omega_p on the D3Q19 half-row kernel (Section 2.2 item 3): the pressure
// (density) update relaxes with omega_p, the momentum with omega. In the moment form
// (lwacm_core.cuh) the density then sums every streamed link value with s_p = 18 nu_p
// in place of s = 18 nu, which adds sdelta = 18 (nu_p - nu) times
//     P(x) = sum_i w_i rho(x - c_i) (c_i . u(x - c_i)) = sum_i w_i c_i . J(x - c_i),
// J = rho u, to the density the plain update forms. P depends on the state at t
// only, so this pass forms it before the step, into a scratch field, and the
// half-row kernel (variant 4) adds sdelta P to each node's density before the
// velocity quotient.
//
// Per axis a, the links with c_a = +1 are e_a (weight 1/18) and e_a + t for the four
// t = +-e_b, b != a (weight 1/36); so with
//     S_a(y) = [2 J_a(y) + sum_{b != a, +-} J_a(y -+ e_b)] / 36
// P(x) = sum_a [S_a(x - e_a) - S_a(x + e_a)]. A block marches a 32 x 16 tile of an
// x-y plane along z, J of three planes (tile plus a one-node frame, wrapped
// periodically) in shared memory (four plane slots, one barrier per plane), the
// loads of the plane after next in flight; the nodes of a last tile beyond nx or ny
// are summed from wrapped ones and not stored.
#include <stdint.h>

#include "launch.h"
#include "lwacm_core.cuh"

namespace lwacm {
namespace {

constexpr int NX_T = 32, NY_T = 16, FX = NX_T + 2, FY = NY_T + 2;
constexpr int NTHR = NX_T * NY_T, PER = (FX * FY + NTHR - 1) / NTHR;  // frame nodes per thread

// zc: planes per block
template <typename T>
__global__ void __launch_bounds__(NTHR) k_nup_sum(const T *__restrict__ in, float *__restrict__ pf, StepParams p,
                                                   int tiles_x, int tiles_y, int zc) {
    __shared__ float J[4][3][FY][FX];  // [plane slot (z mod 4)][component][y][x]
    const int tid = threadIdx.x, tx = tid % NX_T, ty = tid / NX_T;
    const int bt = (int)blockIdx.x % (tiles_x * tiles_y), bz = (int)blockIdx.x / (tiles_x * tiles_y);
    const int x0 = (bt % tiles_x) * NX_T, y0 = (bt / tiles_x) * NY_T;
    const int za = bz * zc, zb = za + zc < p.nz ? za + zc : p.nz;
    const long long plane = (long long)p.nx * p.ny;
    const T *D = in, *U = in + p.fstride, *V = in + 2 * p.fstride, *W = in + 3 * p.fstride;

    // the frame nodes of this thread (tile plus a one-node frame, wrapped), as
    // in-plane offsets: the loads of plane z + 2 are issued before plane z is
    // summed, so that they are in flight meanwhile
    long long off[PER];
    int fpos[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int k = tid + q * NTHR;
        const int fy = k / FX, fx = k - fy * FX;
        // wrapped by a remainder: the frame of a ragged last tile may reach past 2 ny
        const int x = (x0 - 1 + fx + p.nx) % p.nx, y = (y0 - 1 + fy + p.ny) % p.ny;
        off[q] = (long long)y * p.nx + x;
        fpos[q] = k < FX * FY ? k : -1;
    }
    float r[PER][4];
    auto fetch = [&](int z) {
        const long long zo = (long long)(z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z)) * plane;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            if (fpos[q] < 0) continue;
            const long long o = zo + off[q];
            r[q][0] = ldf(D + o);
            r[q][1] = ldf(U + o);
            r[q][2] = ldf(V + o);
            r[q][3] = ldf(W + o);
        }
    };
    auto put = [&](int s) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            if (fpos[q] < 0) continue;
            const int fy = fpos[q] / FX, fx = fpos[q] - fy * FX;
            const float rho = 1.f + r[q][0];
            J[s][0][fy][fx] = rho * r[q][1];
            J[s][1][fy][fx] = rho * r[q][2];
            J[s][2][fy][fx] = rho * r[q][3];
        }
    };
    // four slots: while planes z - 1, z, z + 1 are read, plane z + 2 goes into the
    // fourth, so one barrier per plane suffices
    fetch(za - 1);
    put(3);
    fetch(za);
    put(0);
    fetch(za + 1);
    put(1);
    if (za + 1 < zb) fetch(za + 2);
    __syncthreads();
    int sm = 3, s0 = 0, sp = 1, sn = 2;
    const int cx = tx + 1, cy = ty + 1;
    const float k36 = 1.f / 36.f;
    for (int z = za; z < zb; ++z) {
        if (z + 1 < zb) put(sn);  // plane z + 2, fetched one iteration ago
        if (z + 2 < zb) fetch(z + 3);
        // S_x at x -+ 1, S_y at y -+ 1 (plane z), S_z at z -+ 1
        auto sx = [&](int xx) {
            return (2.f * J[s0][0][cy][xx] + J[s0][0][cy - 1][xx] + J[s0][0][cy + 1][xx] + J[sm][0][cy][xx] +
                    J[sp][0][cy][xx]) * k36;
        };
        auto sy = [&](int yy) {
            return (2.f * J[s0][1][yy][cx] + J[s0][1][yy][cx - 1] + J[s0][1][yy][cx + 1] + J[sm][1][yy][cx] +
                    J[sp][1][yy][cx]) * k36;
        };
        auto sz = [&](int s) {
            return (2.f * J[s][2][cy][cx] + J[s][2][cy][cx - 1] + J[s][2][cy][cx + 1] + J[s][2][cy - 1][cx] +
                    J[s][2][cy + 1][cx]) * k36;
        };
        const float P = ((sx(cx - 1) - sx(cx + 1)) + (sy(cy - 1) - sy(cy + 1))) + (sz(sm) - sz(sp));
        if (y0 + ty < p.ny && x0 + tx < p.nx) pf[(long long)z * plane + (long long)(y0 + ty) * p.nx + x0 + tx] = P;
        __syncthreads();  // plane z + 2 is complete; slot sm is written next
        const int t = sm;
        sm = s0;
        s0 = sp;
        sp = sn;
        sn = t;
    }
}

template <typename T>
cudaError_t launch_t(const void *in, float *pf, const StepParams &p, cudaStream_t st) {
    // the last tiles may be short in x and y
    const int tiles_x = (p.nx + NX_T - 1) / NX_T, tiles_y = (p.ny + NY_T - 1) / NY_T;
    const long long tiles = (long long)tiles_x * tiles_y;
    const int zc = 32;  // planes per block (64 measured slower: fewer blocks in flight)
    const long long blocks = tiles * ((p.nz + zc - 1) / zc);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_nup_sum<T><<<(unsigned)blocks, NTHR, 0, st>>>((const T *)in, pf, p, tiles_x, tiles_y, zc);
    return cudaGetLastError();
}

}  // namespace

bool nup_sum_supported(const StepParams &p) { return p.nx >= 1 && p.ny >= 1 && p.nz >= 1; }
static_assert(FX * FY <= PER * NTHR, "every frame node has a thread");

cudaError_t launch_nup_sum(int storage, const void *in, float *pf, const StepParams &p, cudaStream_t st) {
    if (!nup_sum_supported(p) || !pf) return cudaErrorInvalidValue;
    switch (storage) {
        case STORE_F32: return launch_t<float>(in, pf, p, st);
        case STORE_BF16: return launch_t<__nv_bfloat16>(in, pf, p, st);
        case STORE_F16: return launch_t<__half>(in, pf, p, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lwacm
