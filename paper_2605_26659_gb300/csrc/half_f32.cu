// Half-step kernels on absolute levels, float32 log-domain plans.
#include "half_launch.cuh"

namespace finom {
FINOM_HALF_INST(float)
}  // namespace finom
