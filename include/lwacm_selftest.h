/*
 * lwacm_selftest.h — device self-tests of numerical building blocks the LW-ACM
 * kernels use (the paper has no counterpart). They let a test check, on the
 * GPU, a device function against the hardware's correctly rounded result.
 */
#ifndef LWACM_SELFTEST_H
#define LWACM_SELFTEST_H

#ifdef __cplusplus
extern "C" {
#endif

/* out_dev[k] = the reciprocal 1/x_dev[k] exactly as the row-tiled kernels compute
 * 1/rho for u = j/rho (step a5 of the update): the hardware's approximate
 * reciprocal refined by one Newton-Raphson step, r <- r + r (1 - x r).
 * x_dev, out_dev: caller-owned device arrays of n FP32 values; n in [1, 2^31).
 * Stream-ordered on `stream` (cudaStream_t; NULL = legacy default stream), not
 * synchronised. Errors: LWACM_E_ARG (null pointer, n out of range), LWACM_E_CUDA
 * (launch failure). Return values are lwacm_status codes (lwacm.h). */
int lwacm_selftest_reciprocal(const float *x_dev, float *out_dev, long long n, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LWACM_SELFTEST_H */
