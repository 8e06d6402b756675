// Instantiations of the fused half-step kernel with smaller tiles (1, 2 or
// 4 points per thread) for the launch modes of 1D plans (products, the half
// steps of the loop, the loop-head check, the tile-map pass) and of batches.
#include "apply_launch.cuh"

namespace finom {

template <class R, int E>
static bool launch_e(cudaLaunchConfig_t& cfg, const ApplyArgs<R>& a, int mode, int64_t units, size_t smem,
                     cudaError_t* e) {
  switch (mode) {
    case kModeAgg: *e = launch_mode<R, kModeAgg, E>(cfg, a, units, smem); return true;
    case kModeHalfY: *e = launch_mode<R, kModeHalfY, E>(cfg, a, units, smem); return true;
    case kModeHalfX: *e = launch_mode<R, kModeHalfX, E>(cfg, a, units, smem); return true;
    case kModeCheck: *e = launch_mode<R, kModeCheck, E>(cfg, a, units, smem); return true;
    case kModeLin: *e = launch_mode<R, kModeLin, E>(cfg, a, units, smem); return true;
    case kModeLog: *e = launch_mode<R, kModeLog, E>(cfg, a, units, smem); return true;
    case kModeBHalfY: *e = launch_mode<R, kModeBHalfY, E>(cfg, a, units, smem); return true;
    case kModeBHalfX: *e = launch_mode<R, kModeBHalfX, E>(cfg, a, units, smem); return true;
    case kModeBAgg: *e = launch_mode<R, kModeBAgg, E>(cfg, a, units, smem); return true;
    case kModeBCheck: *e = launch_mode<R, kModeBCheck, E>(cfg, a, units, smem); return true;
    default: return false;
  }
}

template <>
bool launch_apply_small<FINOM_SMALL_R>(cudaLaunchConfig_t& cfg, const ApplyArgs<FINOM_SMALL_R>& a, int mode,
                                       int64_t units, size_t smem, cudaError_t* e) {
  switch (a.elems) {
    case 1: return launch_e<FINOM_SMALL_R, 1>(cfg, a, mode, units, smem, e);
    case 2: return launch_e<FINOM_SMALL_R, 2>(cfg, a, mode, units, smem, e);
    case 4: return launch_e<FINOM_SMALL_R, 4>(cfg, a, mode, units, smem, e);
    default: return false;
  }
}

}  // namespace finom
