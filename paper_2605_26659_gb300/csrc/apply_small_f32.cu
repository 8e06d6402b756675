// Smaller-tile half-step kernels, float32 log-domain plans.
#define FINOM_SMALL_R float
#include "apply_small.cuh"
