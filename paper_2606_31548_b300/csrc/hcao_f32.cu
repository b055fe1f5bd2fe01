// FP32-mode kernels: velocities, relative speeds and the LB sampler in FP32,
// energy bookkeeping, reaction thresholds and reductions in FP64.
#include "hcao_kernels.cuh"

namespace hcao {
HCAO_INSTANTIATE(float)
}  // namespace hcao
