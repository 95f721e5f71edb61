// Internal host-side interface between the C-ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>

namespace lwacm {

struct StepParams;

// storage / transfer element types (same values as the public LWACM_* codes)
enum { STORE_F32 = 0, STORE_BF16 = 1, STORE_F16 = 2 };
enum { XFER_F32 = 0, XFER_F64 = 3 };

constexpr int kDiagBlocks = 152 * 2;  // fixed grid -> deterministic reduction order
constexpr int kDiagValues = 9;

cudaError_t launch_step_generic(int Q, int storage, const void *in, void *out,
                                const StepParams &p, cudaStream_t st);
cudaError_t launch_wall_pass(int Q, int storage, const void *in, void *out, const StepParams &p,
                             cudaStream_t st);
long long wall_node_count(const StepParams &p, int Q);
cudaError_t launch_convert_in(int storage, int src_dtype, const void *src, void *dst, long long n,
                              cudaStream_t st);
cudaError_t launch_convert_out(int storage, int dst_dtype, const void *src, void *dst, long long n,
                               cudaStream_t st);
cudaError_t launch_diagnostics(int storage, const void *f, long long fstride, long long N,
                               int has_z, double *partial, double *out, cudaStream_t st);

// Tiled interior kernels (periodic axes only). supported_* says whether a shape
// can use them; launch_* runs one step.
bool tiled_supported(int Q, int storage, const StepParams &p);
cudaError_t launch_step_tiled(int Q, int storage, const void *in, void *out, const StepParams &p,
                              cudaStream_t st);
const char *tiled_name(int Q);

// Adjoint of one step (periodic; kernels_adjoint.cu): lambda_t from lambda_t1, the
// states at t and t+1; dj is scratch for (Dbar, Jbar); adds dL/dnu to *nu_total.
int adjoint_partials();
cudaError_t launch_adjoint_step(int Q, const float *state_t, const float *state_t1, const float *lam_t1,
                                float *dj, float *lam_t, const StepParams &p, double *nu_partial,
                                double *nu_total, cudaStream_t st);

// Register-prefetch z-marching variant of the D3Q19 kernel (same shapes).
bool zmarch_supported(int Q, int storage, const StepParams &p);
cudaError_t launch_step_zmarch(int Q, int storage, const void *in, void *out, const StepParams &p,
                               cudaStream_t st);

}  // namespace lwacm
