/*
 * lwacm_selftest.h — device self-tests of numerical building blocks the LW-ACM
 * kernels use (the paper has no counterpart). They let a test check, on the
 * GPU, a device function against the correctly rounded result.
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

#ifdef __cplusplus
}
#endif

#endif /* LWACM_SELFTEST_H */
