// Internal host-side interface between the C-ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>

#include <string>

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
// semi-implicit density pass (Eq. FDcompact_si) after the explicit step in -> out
cudaError_t launch_semi_implicit(int Q, int storage, const void *in, void *out, const StepParams &p,
                                 cudaStream_t st);
cudaError_t launch_convert_in(int storage, int src_dtype, const void *src, void *dst, long long n,
                              cudaStream_t st);
cudaError_t launch_convert_out(int storage, int dst_dtype, const void *src, void *dst, long long n,
                               cudaStream_t st);
cudaError_t launch_diagnostics(int storage, const void *f, long long fstride, long long N,
                               int has_z, double *partial, double *out, cudaStream_t st);

// Adjoint of one step (kernels_adjoint.cu) from the states at t and t+1 and
// (Dbar, Jbar) in dj; adds dL/dnu to *nu_total. With lam_t1 (the first step of a
// sweep), dj is first formed from lambda_t1 and the state at t+1. With dj_next, the
// step writes (Dbar, Jbar) of the next step (t-1) there; otherwise lambda_t to
// lam_t. `done` is a zeroed counter the step leaves zeroed.
int adjoint_partials();
cudaError_t launch_adjoint_step(int Q, const float *state_t, const float *state_t1, const float *lam_t1,
                                float *dj, float *dj_next, float *lam_t, const StepParams &p, double *nu_partial,
                                unsigned *done, double *nu_total, cudaStream_t st);

// Batched independent periodic domains packed in one set of field arrays
// (kernels_batch.cu). A tile is batch_tile() consecutive nodes of one domain.
struct BatchDomain {
    int nx, ny, nz, pad;
    long long off, n;  // first node (packed index) and node count
    float s, a;        // 18 nu and 1 - 6 nu of this domain
};
struct BatchTile {
    int dom, pad;
    long long start;   // packed index of the tile's first node
};
// 2D tile of a D2Q9 domain: interior nodes [x0, x0 + TW) x [y0, y0 + TH) (clipped
// to the domain), for the tile shapes of batch_shape()
struct BatchTile2 {
    int dom, x0, y0, pad;
};
struct BatchParams {
    const BatchDomain *doms;
    const BatchTile *tiles;
    const BatchTile2 *tiles2;  // same storage as tiles, used when shape > 0
    int shape;                 // 0: 1D tiles of batch_tile() nodes; k > 0: 2D shape k
    long long ntiles;
    long long fstride;
    unsigned *bar_count;  // followed by the barrier generation word
    unsigned *bar_gen;
    int *err;
    long long withhold_step;  // test hook: CTA 0 skips the barrier after this step (-1: never)
};
int batch_tile();
// 2D tile shapes of the D2Q9 batched kernel (interior width x height); shape 0 is
// the 1D tiling. batch_shapes() is the number of shapes including 0.
int batch_shapes();
void batch_shape(int k, int *tw, int *th);
bool batch_shape_supported(int Q, int storage, int k);
// the same 2D-tile update for one D2Q9 domain (any boundary, the wall rule applied
// in the kernel; no forcing)
bool tiles2d_supported(int Q, int storage, const StepParams &p);
cudaError_t launch_step_tiles2d(int Q, int storage, int shape, const void *in, void *out, const StepParams &p,
                                cudaStream_t st);
cudaError_t launch_batch_step(int Q, int storage, const void *in, void *out, const BatchParams &bp,
                              cudaStream_t st);
cudaError_t launch_batch_persistent(int Q, int storage, void *buf0, void *buf1, const BatchParams &bp,
                                    long long nsteps, int parity, cudaStream_t st);

// Autotuner cache (tune_cache.cu): the configuration measured fastest for a key.
struct TuneChoice {
    int kernel = 0, tile = 0, mode = 0;
    double us = 0.0;  // microseconds per step when measured
};
bool tune_cache_lookup(const char *path, const std::string &key, TuneChoice *out);
bool tune_cache_store(const char *path, const std::string &key, const TuneChoice &ch);

// Half-row TMA D3Q19 kernel (nx = 256: two warps per row, 16 warps per CTA; nx = 128:
// one warp per row).
bool half_supported(int Q, int storage, const StepParams &p);
// the passive scalar (Eq. ACM2.0t) on its own row-tiled D3Q19 kernel (FP32,
// periodic, nx 128 / 256, ny % 8 == 0), run after the flow kernel on the same state
bool scalar_rows_supported(int Q, int storage, const StepParams &p);
cudaError_t launch_scalar_rows(const void *in, void *out, const StepParams &p, cudaStream_t st);
// whether the half-row kernel applies the x-face walls itself (the wall pass then
// leaves the inner x-face nodes alone)
bool half_xwalls(const StepParams &p);
// omega_p on the half-row kernel: P(x) = sum_i w_i c_i . J(x - c_i) of the state `in`
// (FP32, one value per node) into pf, before the step
bool nup_sum_supported(const StepParams &p);
cudaError_t launch_nup_sum(int storage, const void *in, float *pf, const StepParams &p, cudaStream_t st);
// stochastic rounding: advance the step counter the next step's random key is drawn from
cudaError_t launch_sr_tick(unsigned *ctr, cudaStream_t st);
cudaError_t launch_step_half(int Q, int storage, const void *in, void *out, const StepParams &p,
                             cudaStream_t st);

}  // namespace lwacm
