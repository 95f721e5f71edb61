/*
 * lwacm_measure.h — machine measurement used to place the LW-ACM kernels on a
 * roofline (the paper has no counterpart; Section 2.4 and Table performance
 * discuss whether the method is memory- or arithmetic-bound, which is the
 * question this answers on the running GPU).
 */
#ifndef LWACM_MEASURE_H
#define LWACM_MEASURE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Measured single-precision FMA throughput of the current CUDA device.
 *
 * Launches a register-only kernel (eight independent FP32 fused multiply-add
 * chains per thread, 32 warps per SM on every SM, `iters` rounds of 128 FMAs per
 * thread) once to warm up and once timed with CUDA events on `stream`
 * (cudaStream_t; NULL = legacy default stream), and waits for it. Writes the
 * achieved rate in TFLOP/s (2 flops per FMA) to *tflops and the timed launch's
 * duration in milliseconds to *ms. It allocates no device memory (the kernel's
 * only store goes to a 4-byte array inside the library, and only when the chain
 * values meet a condition they never meet for the fixed inputs).
 *
 * iters must lie in [1, 1<<20]; about 4096 gives a launch of a few milliseconds.
 * Errors: LWACM_E_ARG (null output pointer, iters out of range), LWACM_E_CUDA
 * (launch or event failure). Return values are lwacm_status codes (lwacm.h). */
int lwacm_measure_fp32_peak(long long iters, void *stream, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* LWACM_MEASURE_H */
