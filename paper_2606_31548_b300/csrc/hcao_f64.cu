// FP64 parity-mode kernels.  Built with -fmad=false: every floating-point
// expression is evaluated in the written order without FMA contraction, so the
// integer decisions match an IEEE-754 double CPU evaluation bit for bit.
#define HCAO_COMMON_KERNELS 1
#include "hcao_kernels.cuh"

namespace hcao {
HCAO_INSTANTIATE(double)
}  // namespace hcao
