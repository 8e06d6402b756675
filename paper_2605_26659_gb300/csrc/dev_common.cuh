// Device-side building blocks shared by the kernels: the PTX base-2
// exponential and logarithm, warp and block reductions, and programmatic
// dependent launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace finom {

// 2^x and log2 x by the PTX approximations (ex2.approx: relative error
// about 2^-22.5; lg2.approx: absolute error about 2^-22)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// exclusive block sum of one int per thread
template <int NT>
__device__ __forceinline__ int block_exclusive_sum(int v, int* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  int wp = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w)
    if (w < warp) wp += sh[w];
  __syncthreads();
  return wp + inc - v;
}

// programmatic dependent launch: wait until the previous kernel of the
// stream has completed and its writes are visible; allow the next kernel of
// the stream to be scheduled (its blocks start as ours exit).  Both are
// no-ops when the launch did not ask for programmatic serialisation.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

}  // namespace finom
