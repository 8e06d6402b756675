// Plan construction: merged order of the two meshes, dividing indices, gaps.
//
// The dividing index (Definition, Sec. 2.2) is zeta(i) = #{j : y_j <= x_i};
// for K^T the same definition with the meshes swapped gives
// zetaT(j) = #{i : x_i <= y_j}.  Merging both meshes with y before x on ties
// puts x_i at merged position i + zeta(i) and y_j at j + #{i : x_i < y_j}.
// Between consecutive merged points the kernel factor is
// 2^{-gap_k}, gap_k = (z_k - z_{k-1}) / (eps ln 2): the ratio vectors r, r'
// of the Theorems on the vector representation of K_L and K_U (eq. ratio)
// are products of these factors over the merged points between two rows.
//
// The merge is a merge path: one binary search on the diagonal k0 of every
// tile boundary gives the x points among the first k0 merged points; each
// tile then stages its x and y runs in shared memory, every thread finds
// its own diagonal inside the tile the same way and merges its points
// serially, writing the type bits, the gaps and the dividing index of its x
// points.  Every point is read once from global memory.
#include <cuda_runtime.h>

#include <string>

#include <cmath>
#include <vector>

#include "dev_common.cuh"
#include "finom_internal.h"

namespace finom {

namespace {

__global__ void k_check_sorted(const double* a, int64_t n, int* bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = a[i];
  bool ok = isfinite(v);
  if (i + 1 < n) ok = ok && (v <= a[i + 1]);
  if (!ok) atomicOr(bad, 1);
}

// x points among the first d merged points (y before x on ties): the
// number of k with pos(x_k) < d, i.e. with x_k before y_{d-k-1}, found by
// bisection on the diagonal i + j = d
__device__ __forceinline__ int64_t merge_split(const double* x, int64_t N, const double* y, int64_t M,
                                               int64_t d) {
  int64_t lo = d > M ? d - M : 0, hi = d < N ? d : N;
  while (lo < hi) {   // for lo <= k < hi: 0 <= d - k - 1 < M
    const int64_t k = (lo + hi) >> 1;
    if (x[k] < y[d - k - 1]) lo = k + 1; else hi = k;
  }
  return lo;
}

// tile_x0[t] = x points among the first min(t * kTile, L) merged points
__global__ void k_tile_split(const double* x, int64_t N, const double* y, int64_t M, int64_t C,
                             int32_t* tile_x0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t > C) return;
  tile_x0[t] = (int32_t)merge_split(x, N, y, M, min(t * (int64_t)kTile, N + M));
}

// One CTA per tile of kTile merged points, kElems per thread: type bits,
// gaps in bits (gap64) and zeta of the tile's x points.
__global__ void __launch_bounds__(kThreads) k_merge(const double* x, int64_t N, const double* y, int64_t M,
                                                    const int32_t* tile_x0, double inv_eps_ln2, int32_t* zeta,
                                                    double* gap64, uint32_t* bits) {
  __shared__ double sx[kTile], sy[kTile];
  const int tid = threadIdx.x;
  const int64_t L = N + M;
  const int64_t k0 = (int64_t)blockIdx.x * kTile;
  const int64_t kend = min(k0 + (int64_t)kTile, L);
  const int64_t x0 = tile_x0[blockIdx.x], x1 = tile_x0[blockIdx.x + 1];
  const int64_t y0 = k0 - x0, y1 = kend - x1;
  const int nx = (int)(x1 - x0), ny = (int)(y1 - y0);
  for (int i = tid; i < nx; i += kThreads) sx[i] = x[x0 + i];
  for (int j = tid; j < ny; j += kThreads) sy[j] = y[y0 + j];
  __syncthreads();
  // this thread's diagonal inside the tile
  const int dl = tid * kElems;
  uint32_t b8 = 0;
  if (k0 + dl < kend) {
    int lo = dl > ny ? dl - ny : 0, hi = dl < nx ? dl : nx;
    while (lo < hi) {
      const int k = (lo + hi) >> 1;
      if (sx[k] < sy[dl - k - 1]) lo = k + 1; else hi = k;
    }
    int i = lo, j = dl - lo;
    // the merged point before this thread's first one: the later (larger)
    // of the x and y points before the split
    double prev = -INFINITY;
    if (x0 + i > 0) prev = x[x0 + i - 1];
    if (y0 + j > 0) prev = fmax(prev, y[y0 + j - 1]);
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const int64_t k = k0 + dl + e;
      if (k >= kend) break;
      const bool take_x = i < nx && (j >= ny || sx[i] < sy[j]);
      double v;
      if (take_x) {
        v = sx[i];
        zeta[x0 + i] = (int32_t)(y0 + j);   // the y points before x_i
        b8 |= 1u << e;
        ++i;
      } else {
        v = sy[j];
        ++j;
      }
      gap64[k] = k == 0 ? 0.0 : (v - prev) * inv_eps_ln2;
      prev = v;
    }
  }
  // kElems-bit chunks of 32 / kElems consecutive threads form one word
  constexpr int kPer = 32 / kElems;
  uint32_t w = b8 << ((tid % kPer) * kElems);
#pragma unroll
  for (int o = 1; o < kPer; o <<= 1) w |= __shfl_xor_sync(0xffffffffu, w, o);
  if (tid % kPer == 0) bits[(k0 + dl) >> 5] = w;
}

// zetaT(j) = #{i : x_i <= y_j} (the dividing index of K^T, Definition applied
// to K^T; reported by finom_dividing_index only)
__global__ void k_zeta_t(const double* x, int64_t N, const double* y, int64_t M, int32_t* zetaT) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double v = y[j];
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (x[mid] <= v) lo = mid + 1; else hi = mid;
  }
  zetaT[j] = (int32_t)lo;
}

// the same table for tiles of `tile` points from the dividing index: the
// merged position of x_i is i + zeta(i) (y before x on ties), increasing in i
__global__ void k_tiles_zeta(const int32_t* zeta, int64_t N, int64_t C, int64_t tile, int32_t* tile_x0) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t > C) return;
  const int64_t bound = t * tile;
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (mid + (int64_t)zeta[mid] < bound) lo = mid + 1; else hi = mid;
  }
  tile_x0[t] = (int32_t)lo;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

finom_status build_plan(finom_plan_s* p, const double* x, const double* y, cudaStream_t s) {
  const int64_t N = p->N, M = p->M, L = N + M;
  p->L = L;
  p->C = (L + kTile - 1) / kTile;
  // tile-aligned sizes: every tile writes its whole words of type bits, and
  // vector loads past L stay inside the allocations
  const int64_t Lpad = p->C * kTile;

  FINOM_CUDA(cudaMalloc(&p->x, sizeof(double) * N));
  FINOM_CUDA(cudaMalloc(&p->y, sizeof(double) * M));
  FINOM_CUDA(cudaMemcpyAsync(p->x, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  FINOM_CUDA(cudaMemcpyAsync(p->y, y, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));

  int* bad = nullptr;
  FINOM_CUDA(cudaMalloc(&bad, sizeof(int)));
  FINOM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_check_sorted<<<nblk(N, 256), 256, 0, s>>>(p->x, N, bad);
  k_check_sorted<<<nblk(M, 256), 256, 0, s>>>(p->y, M, bad);
  int hbad = 0;
  FINOM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  cudaFree(bad);
  if (hbad) {
    set_error("finom_plan: x and y must be finite and sorted non-decreasing");
    return FINOM_EINVAL;
  }

  FINOM_CUDA(cudaMalloc(&p->zeta, sizeof(int32_t) * N));
  FINOM_CUDA(cudaMalloc(&p->zetaT, sizeof(int32_t) * M));
  FINOM_CUDA(cudaMalloc(&p->tbits, sizeof(uint32_t) * (Lpad / 32)));
  FINOM_CUDA(cudaMalloc(&p->gap64, sizeof(double) * Lpad));
  FINOM_CUDA(cudaMemsetAsync(p->gap64, 0, sizeof(double) * Lpad, s));
  FINOM_CUDA(cudaMalloc(&p->tile_x0, sizeof(int32_t) * (p->C + 1)));
  const double inv = 1.0 / (p->eps * std::log(2.0));
  k_tile_split<<<nblk(p->C + 1, 256), 256, 0, s>>>(p->x, N, p->y, M, p->C, p->tile_x0);
  k_merge<<<(unsigned)p->C, kThreads, 0, s>>>(p->x, N, p->y, M, p->tile_x0, inv, p->zeta, p->gap64, p->tbits);
  k_zeta_t<<<nblk(M, 256), 256, 0, s>>>(p->x, N, p->y, M, p->zetaT);
  FINOM_CUDA(cudaGetLastError());
  FINOM_CUDA(cudaStreamSynchronize(s));
  p->elems = kElems;
  p->Ce = p->C;
  p->tile_x0e = p->tile_x0;
  return FINOM_OK;
}

finom_status build_tiles_e(finom_plan_s* p, int elems, cudaStream_t s) {
  if (!tile_kind_ok(elems)) {
    set_error("tile kind must be 1, 2, 4 or " + std::to_string(kElems) + " points per thread, or " +
              std::to_string(kElemsSmall) + " (64-point tiles)");
    return FINOM_EINVAL;
  }
  if (elems == p->elems) return FINOM_OK;
  if (p->tile_x0e && p->tile_x0e != p->tile_x0) cudaFree(p->tile_x0e);
  p->tile_x0e = p->tile_x0;
  p->Ce = p->C;
  p->elems = kElems;
  if (elems == kElems) return FINOM_OK;
  const int64_t tile = tile_points(elems);
  const int64_t Ce = (p->L + tile - 1) / tile;
  int32_t* t0 = nullptr;
  FINOM_CUDA(cudaMalloc(&t0, sizeof(int32_t) * (Ce + 1)));
  k_tiles_zeta<<<nblk(Ce + 1, 256), 256, 0, s>>>(p->zeta, p->N, Ce, tile, t0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(t0);
    return cuda_fail(e, "k_tiles_zeta");
  }
  p->tile_x0e = t0;
  p->Ce = Ce;
  p->elems = elems;
  return FINOM_OK;
}

void free_plan(finom_plan_s* p) {
  cudaFree(p->x);
  cudaFree(p->y);
  cudaFree(p->zeta);
  cudaFree(p->zetaT);
  cudaFree(p->tbits);
  cudaFree(p->gap64);
  if (p->tile_x0e && p->tile_x0e != p->tile_x0) cudaFree(p->tile_x0e);
  cudaFree(p->tile_x0);
}

}  // namespace finom
