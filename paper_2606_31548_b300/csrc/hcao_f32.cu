// FP32-mode kernels: velocities, relative speeds and the LB sampler in FP32,
// energy bookkeeping, reaction thresholds and reductions in FP64.
#include "hcao_kernels.cuh"
#include "hcao_fused.cuh"

namespace hcao {
HCAO_INSTANTIATE(float)
}  // namespace hcao
