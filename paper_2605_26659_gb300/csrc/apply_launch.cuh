// Host-side launch helpers of the fused half-step kernel, shared by the
// translation units that instantiate it (apply.cu: the full tile of kElems
// points per thread for every mode; apply_small_*.cu: smaller tiles for the
// modes of 1D plans).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "apply.cuh"
#include "finom_internal.h"

namespace finom {

// persistent grid: as many CTAs as fit on the device at once, at most one per unit
template <class R, int M, int E>
unsigned grid_of(int64_t units, size_t smem) {
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_apply<R, M, E>, kThreads, smem) != cudaSuccess) n = 1;
    per_sm = n < 1 ? 1 : n;
  }
#ifndef FINOM_PERSIST
#define FINOM_PERSIST 1
#endif
  return (unsigned)(FINOM_PERSIST ? std::min<int64_t>(units, (int64_t)per_sm * sms) : units);
}

template <class R, int M, int E>
cudaError_t launch_mode(cudaLaunchConfig_t& cfg, const ApplyArgs<R>& a, int64_t units, size_t smem) {
  cfg.gridDim = dim3(grid_of<R, M, E>(units, smem));
  return cudaLaunchKernelEx(&cfg, k_apply<R, M, E>, a);
}

// launches a 1D-plan mode with a.elems points per thread (1, 2 or 4); false
// if that mode or tile size is not instantiated
template <class R>
bool launch_apply_small(cudaLaunchConfig_t& cfg, const ApplyArgs<R>& a, int mode, int64_t units, size_t smem,
                        cudaError_t* e);

}  // namespace finom
