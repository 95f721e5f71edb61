// Tiled interior kernels (placeholder until the z-marching kernel lands).
#include "launch.h"
#include "lwacm_core.cuh"

namespace lwacm {

bool tiled_supported(int, int, const StepParams &) { return false; }
cudaError_t launch_step_tiled(int, int, const void *, void *, const StepParams &, cudaStream_t) {
    return cudaErrorNotSupported;
}
const char *tiled_name(int Q) { return Q == 9 ? "tiled_d2q9" : "tiled_d3q19"; }

}  // namespace lwacm
