// Building blocks of the row-tiled D3Q19 kernels (kernels_half.cu, kernels_scalar.cu)
// and their self-tests (selftest.cu): per-launch parameters, mbarrier / bulk-copy
// wrappers, the correctly rounded velocity quotient, the work schedule (planned on
// the host, iterated on the device and on the host) over (y-column, run of planes)
// items, exchange-row slots and storage-type loads and stores.
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
    int ycols;           // columns of ROWS rows: ceil(ny / ROWS)
    int segs;            // 128-node segments per row a CTA item covers one of (1: the whole row)
    int zc, nitems;      // planes per chunk, ycols * ceil(nz / zc); zc = 0: equal runs (TaskIter)
    int kcls;            // equal runs: y-neighbouring columns lie kcls apart in the run order
    long long fstride;
    float s18;           // s / 18 = nu
    float a, am1;        // a = 1 - 6 nu and a - 1 = -6 nu (post_combine, lwacm_core.cuh)
    float g[3];          // constant acceleration of Eq. force (used by the forced variant)
    const unsigned *sr_ctr;  // stochastic rounding (BF16 / FP16 storage): the step counter
    const float *pfield;     // omega_p: sum_i w_i c_i . J(x - c_i) per node (k_nup_sum)
    float sdelta;            // omega_p: 18 (nu_p - nu)
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
// bring `bytes` (a multiple of 16, 16-byte aligned) of global memory into L2
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            sa(dst)),
        "l"(src), "r"(bytes), "r"(sa(bar))
        : "memory");
}

// ---- velocity u = j / rho (step a5: IEEE division) -------------------------------
// The three momentum components of a node share one divisor. Each quotient is the
// correctly rounded one (the IEEE round-to-nearest quotient j / rho), formed with
// Markstein's FMA correction (P. W. Markstein, "Computation of elementary functions
// on the IBM RISC System/6000 processor", IBM J. Res. Develop. 34 (1990) 111-119):
// with y = RN(1/b), the correctly rounded reciprocal (rcp_rn below), and q within
// one ulp of a/b, the residual r = a - b q is exact in one FMA and
// RN(q + r y) = RN(a/b). In brief:
// q + r y misses a/b by (a/b - q)(b y - 1); when a/b lies within 2^-24 ulp of a
// rounding midpoint every faithful q is about half an ulp from a/b, so the miss is
// below half an ulp times |b y - 1| < 2^-24, less than a/b's distance to any
// midpoint (at least 2^-24 ulp / b, as a - b m is a nonzero multiple of a fixed
// power of two).
// The first product q0 = RN(a y) can miss by up to about 1.5 ulps (a near 2 in its
// binade, a/b just below the next), so a first correction q1 = RN(q0 + r0 y) brings
// it within half an ulp plus a few 2^-24 ulp (faithful) and a second correction
// gives the correctly rounded quotient. This holds while the residuals stay normal:
// numerators |a| >= 2^-100 and normal quotients (a smaller momentum, far below any
// resolved velocity, may round one unit differently in the last place). A zero
// numerator gives +0 (the exact residual of a zero quotient is +0), where IEEE
// division keeps the quotient's sign of zero; the two zeros compare equal, and the
// sign of a zero velocity changes no later value of the update.
// Why the rounding matters here: a quotient through a rounded reciprocal and a
// product (two roundings) drifts 1.7e-5 u0 from the FP64 oracle over 1000 steps of
// the 128^3 Taylor-Green workload, the IEEE quotient 4.7e-6 u0. The reciprocal's
// rounding error depends only on the slowly moving density, so it keeps its sign
// at a node over many steps (as in post_combine of lwacm_core.cuh).
// RN(1/b) without branches, for normal b with a normal reciprocal: the hardware's
// approximate reciprocal (relative error far below 2^-20), then two Newton-Raphson
// steps y <- y + y (1 - b y), each an FMA residual and an FMA update. The first
// brings y within one ulp; from there Markstein's reciprocal theorem (same paper)
// makes the second step return RN(1/b) for every b whose significand is not all
// ones. For those, b = (2 - 2^-23) 2^k, 1/b lies just above the midpoint between
// 2^(-k-1) and its successor, which the step rounds to even: one ulp low. RN(1/b)
// then has the last significand bit set, so that bit is set for them.
__device__ __forceinline__ float rcp_approx(float b) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(b));
    return y;
}
__device__ __forceinline__ float rcp_fix(float b, float y) {
    const unsigned ones = ((__float_as_uint(b) & 0x7fffffu) + 1u) >> 23;  // 1 iff significand all ones
    return __uint_as_float(__float_as_uint(y) | ones);
}
__device__ __forceinline__ float rcp_rn(float b) {
    float y = rcp_approx(b);
    y = fmaf(y, fmaf(-b, y, 1.f), y);
    y = fmaf(y, fmaf(-b, y, 1.f), y);
    return rcp_fix(b, y);
}

struct Div1 {
    float nb, y;  // -divisor, RN(1 / divisor)
};
__device__ __forceinline__ Div1 div_prep(float b) {
    Div1 d;
    d.nb = -b;
    d.y = rcp_rn(b);
    return d;
}
__device__ __forceinline__ float div_apply(float a, const Div1 &d) {
    const float q0 = a * d.y;
    const float q1 = fmaf(fmaf(d.nb, q0, a), d.y, q0);  // faithful
    return fmaf(fmaf(d.nb, q1, a), d.y, q1);             // correctly rounded
}
// the same for two nodes held as an FP32x2 pair (packed FMAs, same rounding)
struct Div2 {
    float2 nb, y;
};
__device__ __forceinline__ Div2 div_prep2(float2 b) {
    Div2 d;
    d.nb = make_float2(-b.x, -b.y);
    const float2 one = make_float2(1.f, 1.f);
    float2 y = make_float2(rcp_approx(b.x), rcp_approx(b.y));
    y = __ffma2_rn(y, __ffma2_rn(d.nb, y, one), y);
    y = __ffma2_rn(y, __ffma2_rn(d.nb, y, one), y);
    d.y = make_float2(rcp_fix(b.x, y.x), rcp_fix(b.y, y.y));
    return d;
}
__device__ __forceinline__ float2 div_apply2(float2 a, const Div2 &d) {
    const float2 q0 = __fmul2_rn(a, d.y);
    const float2 q1 = __ffma2_rn(__ffma2_rn(d.nb, q0, a), d.y, q0);
    return __ffma2_rn(__ffma2_rn(d.nb, q1, a), d.y, q1);
}

// ---- task iteration -------------------------------------------------------------
// An item is a run [za, zb) of planes of one column, processed as source planes
// za-1 (FIRST), za .. zb-1 (MID), zb (LAST). Two schedules:
// * chunks (zc > 0): items are (column, z-chunk of zc planes) pairs, numbered
//   chunk-major (item = chunk * ycols + col) so that the CTAs working on
//   neighbouring columns march through the same planes together and share their
//   halo rows in L2; CTA b takes items b, b + G, b + 2G, ... (G = grid size).
// * equal runs (zc == 0): the columns' planes laid end to end (W = ycols nz planes) are
//   cut into G equal runs, CTA b taking planes [b W / G, (b+1) W / G): one or two
//   items (more when a run is longer than a column), the column changing inside a
//   run. Columns follow each other in an order where y-neighbours lie kcls apart:
//   kcls = ycols / gcd(ycols, G) columns hold exactly an integer number of runs, so
//   a column and the one kcls after it start their runs at the same planes, and
//   their CTAs pass each plane together as with chunks.
enum { FIRST = 0, MID = 1, LAST = 2 };

struct TaskIter {
    int item, nitems, stride, ycols, zc, nz;
    // chunks: the item's column and chunk, and the steps of both per item (no
    // division once started)
    int ch, dcol, dch;
    // runs: the next plane of the run and its end; the column's place in the run
    // order (class r, index q in the class) and the columns per class
    long long lin, lend;
    int r, q, kcls, per;
    int col, za, zb, pz;
    __host__ __device__ TaskIter(int first, int nitems_, int stride_, int ycols_, int zc_, int nz_, int kcls_ = 1)
        : item(first), nitems(nitems_), stride(stride_), ycols(ycols_), zc(zc_), nz(nz_), kcls(kcls_) {
        col = za = zb = pz = ch = dcol = dch = r = q = per = 0;
        lin = lend = 0;
        if (zc > 0) {
            dcol = stride % ycols;
            dch = stride / ycols;
            col = item % ycols;
            ch = item / ycols;
        } else {
            const long long w = (long long)ycols * nz;
            lin = w * first / stride;
            lend = w * (first + 1) / stride;
            const int s = (int)(lin / nz);
            za = (int)(lin - (long long)s * nz);
            per = ycols / kcls;
            r = s % kcls;
            q = s / kcls;
        }
        if (valid()) start_run();
    }
    __host__ __device__ void start_run() {
        if (zc > 0) {
            za = ch * zc;
            zb = za + zc < nz ? za + zc : nz;
        } else {
            const long long left = lend - lin;
            zb = left < nz - za ? za + (int)left : nz;
            col = r * per + q;
        }
        pz = za - 1;
    }
    __host__ __device__ bool valid() const { return zc > 0 ? item < nitems : lin < lend; }
    __host__ __device__ int mode() const { return pz < za ? FIRST : (pz < zb ? MID : LAST); }
    __host__ __device__ void next() {
        if (pz < zb) {
            ++pz;
        } else if (zc > 0) {
            item += stride;
            col += dcol;
            ch += dch;
            if (col >= ycols) {
                col -= ycols;
                ++ch;
            }
            if (item < nitems) start_run();
        } else {
            lin += zb - za;
            za = 0;  // a run goes on at the start of the next column
            if (++r == kcls) {
                r = 0;
                ++q;
            }
            if (lin < lend) start_run();
        }
    }
};

// The schedule of a step (TaskIter), chosen on the host: cost model = the busiest CTA's planes plus 0.7
// of a plane per item (its FIRST and LAST source planes, each partly computed).
struct Schedule {
    int zc, nitems, kcls, grid;
};
// chunks of zc planes: the zc with the least cost
inline Schedule chunk_schedule(int cols, int nz, int ctas, double *cost) {
    if (ctas < 1) ctas = 1;
    int best = nz;
    double best_t = 1e300;
    for (int zc = (nz < 4 ? nz : 4); zc <= nz; ++zc) {
        const long long items = (long long)cols * ((nz + zc - 1) / zc);
        const long long per = (items + ctas - 1) / ctas;
        const double t = (double)per * (zc + 0.7);
        if (t < best_t - 1e-9) {
            best_t = t;
            best = zc;
        }
    }
    *cost = best_t;
    const int nitems = cols * ((nz + best - 1) / best);
    return Schedule{best, nitems, 1, ctas < nitems ? ctas : nitems};
}
// equal runs over the columns laid end to end
inline Schedule run_schedule(int cols, int nz, int ctas, double *cost) {
    const long long w = (long long)cols * nz;
    const int g = (int)(w < ctas ? w : ctas);
    double worst = 0.0;
    for (int b = 0; b < g; ++b) {
        const long long l0 = w * b / g, l1 = w * (b + 1) / g;
        const long long items = (l1 - 1) / nz - l0 / nz + 1;
        const double t = (double)(l1 - l0) + 0.7 * (double)items;
        worst = t > worst ? t : worst;
    }
    *cost = worst;
    int a = cols, c = g;  // kcls = cols / gcd(cols, g)
    while (c) {
        const int t = a % c;
        a = c;
        c = t;
    }
    return Schedule{0, g, cols / a, g};
}
inline Schedule plan_schedule(int cols, int nz, int ctas) {
    double tc = 0.0, tr = 0.0;
    const Schedule c = chunk_schedule(cols, nz, ctas, &tc);
    const Schedule r = run_schedule(cols, nz, ctas < 1 ? 1 : ctas, &tr);
    return tr < tc - 1e-9 ? r : c;
}

// position of node group h (4 nodes) of lane l inside an exchange row: the 4-float
// groups of all lanes are contiguous, so warp float4 accesses are conflict-free
__device__ __forceinline__ int spos(int l, int h) { return h * 128 + l * 4; }

template <int PM, int P0, int PP>
__device__ __forceinline__ constexpr int pl(int cz) { return cz > 0 ? PP : (cz < 0 ? PM : P0); }

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

// ---- stochastic rounding to BF16 / FP16 storage -----------------------------------
// A value x between the storage type's neighbours lo and hi (|lo| <= |x| < |hi|,
// same sign) is stored as hi with probability (x - lo) / (hi - lo), else as lo, so
// that the stored value is x in expectation: a change per step below half a storage
// ulp accumulates over the steps instead of being rounded away each step. The 16
// random bits per stored value come from a counter-based generator: MurmurHash3's
// 32-bit finalizer (A. Appleby, MurmurHash3, public domain), a bijection of 32-bit
// words, applied to (node index, field pair) xored with a key drawn from the step
// counter; each field takes one half of the word.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__host__ __device__ __forceinline__ uint32_t sr_key(uint32_t step) { return fmix32(step ^ 0x9e3779b9u); }
// the random word of fields 2q (low half) and 2q+1 (high half) of node k
__device__ __forceinline__ uint32_t sr_bits(uint32_t k, uint32_t q, uint32_t key) { return fmix32(((k << 1) | q) ^ key); }

// bfloat16 is the upper half of an FP32: adding r16 to the discarded half carries
// into the kept half with probability (discarded bits) / 2^16
__device__ __forceinline__ uint16_t sr_bf16(float x, uint32_t r16) {
    const uint32_t b = __float_as_uint(x);
    if ((b & 0x7f800000u) == 0x7f800000u) return __bfloat16_as_ushort(__float2bfloat16_rn(x));  // inf, NaN
    return (uint16_t)((b + r16) >> 16);
}
// FP16 in its normal range (2^-14 <= |x| < 2^16): 13 significand bits are dropped,
// so adding 13 random bits there and rounding toward zero carries into the kept
// bits with probability (dropped bits) / 2^13. Below it the FP16 spacing is a fixed
// 2^-24: the fraction of a spacing is formed exactly and compared with the bits.
__device__ __forceinline__ uint16_t sr_f16(float x, uint32_t r16) {
    const uint32_t b = __float_as_uint(x), ex = (b >> 23) & 0xffu;
    if (ex >= 113u && ex <= 142u) return __half_as_ushort(__float2half_rz(__uint_as_float(b + (r16 & 0x1fffu))));
    if (ex < 113u) {
        const uint16_t lb = __half_as_ushort(__float2half_rz(x));
        const float frac = fabsf(x - __half2float(__ushort_as_half(lb))) * 16777216.f;
        return frac * 65536.f > (float)r16 ? (uint16_t)(lb + 1u) : lb;
    }
    return __half_as_ushort(__float2half_rn(x));  // beyond the FP16 range, inf, NaN
}
__device__ __forceinline__ uint16_t sr_round(float x, uint32_t r16, const __nv_bfloat16 *) { return sr_bf16(x, r16); }
__device__ __forceinline__ uint16_t sr_round(float x, uint32_t r16, const __half *) { return sr_f16(x, r16); }

// store four floats rounded stochastically (r: 16 random bits each, in the low half)
template <typename T>
__device__ __forceinline__ void st4_sr(T *p, float a, float b, float c, float d, uint32_t ra, uint32_t rb,
                                       uint32_t rc, uint32_t rd) {
    uint2 r;
    r.x = (uint32_t)sr_round(a, ra & 0xffffu, p) | ((uint32_t)sr_round(b, rb & 0xffffu, p) << 16);
    r.y = (uint32_t)sr_round(c, rc & 0xffffu, p) | ((uint32_t)sr_round(d, rd & 0xffffu, p) << 16);
    *reinterpret_cast<uint2 *>(p) = r;
}

}  // namespace tile
}  // namespace lwacm
