/*
 * lwacm_selftest.h — self-tests of building blocks the LW-ACM kernels use (the
 * paper has no counterpart). They let a test check, on the GPU, a device function
 * against the correctly rounded result, and, on the host, the work schedule the
 * row-tiled kernels follow.
 */
#ifndef LWACM_SELFTEST_H
#define LWACM_SELFTEST_H

#ifdef __cplusplus
extern "C" {
#endif

/* out_dev[k] = a_dev[k] / b_dev[k] exactly as the row-tiled kernels form the
 * velocity u = j / rho (step a5 of the update, after Eq. ACM2.0b: the moments
 * rho u and rho, divided): the correctly rounded reciprocal of the divisor and two
 * FMA corrections of the quotient (Markstein's method), which give the IEEE
 * round-to-nearest quotient for every normal quotient.
 * packed == 1: elements in pairs (2k, 2k+1) through the FP32x2 form of the
 * half-row kernel (an odd last element through the scalar form); packed == 0:
 * every element through the scalar form; packed == 2: out_dev[k] = the
 * reciprocal RN(1 / b_dev[k]) that the quotient divides with (a_dev is not read,
 * but must be a valid pointer).
 * a_dev, b_dev, out_dev: caller-owned device arrays of n FP32 values; n in
 * [1, 2^31). Stream-ordered on `stream` (cudaStream_t; NULL = legacy default
 * stream), not synchronised. Errors: LWACM_E_ARG (null pointer, n out of range,
 * packed not in {0, 1, 2}),
 * LWACM_E_CUDA (launch failure). Return values are lwacm_status codes (lwacm.h). */
int lwacm_selftest_quotient(const float *a_dev, const float *b_dev, float *out_dev, long long n, int packed,
                            void *stream);

/* out_dev[k] = x_dev[k] rounded stochastically to the storage type (LWACM_BF16 or
 * LWACM_F16) exactly as the half-row kernel stores the density of node k in the step
 * whose counter is `step` (LWACM_OPT_STOCHASTIC_ROUNDING), widened back to FP32
 * (exact): one of the two storage values around x, the one further from zero with
 * probability |x - lo| / |hi - lo|. x_dev, out_dev: caller-owned device arrays of n
 * FP32 values, n in [1, 2^31). Stream-ordered on `stream`, not synchronised.
 * Errors: LWACM_E_ARG (null pointer, n out of range, other storage), LWACM_E_CUDA. */
int lwacm_selftest_round(const float *x_dev, float *out_dev, long long n, int storage, unsigned step, void *stream);

/* The work schedule of one step of the row-tiled kernels (the D3Q19 half-row kernel
 * and the scalar kernel), host only (no GPU needed): `cols` columns of rows (times
 * the 128-node segments of a row, where a row has several) and nz planes on `ctas`
 * resident CTAs. Writes *grid (CTAs launched), *zc (planes per chunk; 0 = equal
 * runs: the columns' planes laid end to end, one run per CTA, y-neighbouring columns
 * kcls apart in the run order) and *kcls, and, CTA by CTA in launch order, each
 * item a CTA takes in the order it takes them, as four ints (CTA, column, za, zb):
 * the planes [za, zb) of that column (the kernel reads source planes za-1 .. zb).
 * *count = the number of items; only the first `cap` are written to items (4 cap
 * ints, caller-owned host memory; may be NULL when cap = 0).
 * Errors: LWACM_E_ARG (cols, nz or ctas < 1, cols * nz >= 2^31, a null output
 * pointer, cap < 0, items NULL with cap > 0). */
int lwacm_selftest_schedule(int cols, int nz, int ctas, int *grid, int *zc, int *kcls, int *items, long long cap,
                            long long *count);

#ifdef __cplusplus
}
#endif

#endif /* LWACM_SELFTEST_H */
