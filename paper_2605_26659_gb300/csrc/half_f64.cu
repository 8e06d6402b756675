// Half-step kernels on absolute levels, float64 plans.
#include "half_launch.cuh"

namespace finom {
FINOM_HALF_INST(double)
}  // namespace finom
