// Smaller-tile half-step kernels, float64 plans.
#define FINOM_SMALL_R double
#include "apply_small.cuh"
