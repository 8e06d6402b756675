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

// number of entries of sorted a[0..n) that are <= v (strict = false) or < v (strict = true)
__device__ __forceinline__ int64_t count_le(const double* a, int64_t n, double v, bool strict) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    bool go_right = strict ? (a[mid] < v) : (a[mid] <= v);
    if (go_right) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_ranks_x(const double* x, int64_t N, const double* y, int64_t M, int32_t* zeta,
                          int64_t* posx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t z = count_le(y, M, x[i], false);
  zeta[i] = (int32_t)z;
  posx[i] = i + z;
}

__global__ void k_ranks_y(const double* x, int64_t N, const double* y, int64_t M, int32_t* zetaT,
                          int64_t* posy) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  double v = y[j];
  zetaT[j] = (int32_t)count_le(x, N, v, false);
  posy[j] = j + count_le(x, N, v, true);
}

__global__ void k_scatter(const double* a, int64_t n, const int64_t* pos, double* z, uint8_t* type,
                          uint8_t t) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[pos[i]] = a[i];
  type[pos[i]] = t;
}

// gaps in bits and packed type bits; one thread per merged position, padded to
// a multiple of 32 so every warp writes one whole word.
__global__ void k_gaps_bits(const double* z, const uint8_t* type, int64_t L, double inv_eps_ln2,
                            double* gap64, float* gap32, uint32_t* bits) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool in = k < L;
  int t = in ? (int)type[k] : 0;
  unsigned w = __ballot_sync(0xffffffffu, t != 0);
  if ((threadIdx.x & 31) == 0 && (k >> 5) < ((L + 31) >> 5)) bits[k >> 5] = w;
  if (!in) return;
  double g = (k == 0) ? 0.0 : (z[k] - z[k - 1]) * inv_eps_ln2;
  gap64[k] = g;
  if (gap32) gap32[k] = (float)g;
}

// tile_x0[t] = number of x points whose merged position is < t * kTile
__global__ void k_tiles(const int64_t* posx, int64_t N, int64_t C, int32_t* tile_x0) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t > C) return;
  int64_t bound = t * (int64_t)kTile;
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (posx[mid] < bound) lo = mid + 1; else hi = mid;
  }
  tile_x0[t] = (int32_t)lo;
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

// fw[o_is_x][t]: index of the last W point before the O point that precedes
// tile t (0 when there is none); the O point before the first O point of the
// sequence is that point itself
__global__ void k_frame_w(const double* x, int64_t N, const double* y, int64_t M, const int32_t* zeta,
                          const int32_t* tile_x0, int64_t C, int64_t L, int32_t* fw_y, int32_t* fw_x) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t > C) return;
  const int64_t k0 = min(t * (int64_t)kTile, L);
  const int64_t x0 = tile_x0[t], y0 = k0 - x0;
  // O = x: W points before x_o are the y_j <= x_o
  const int64_t ox = x0 > 0 ? x0 - 1 : 0;
  fw_x[t] = (int32_t)max((int64_t)zeta[ox] - 1, (int64_t)0);
  // O = y: W points before y_o are the x_i < y_o
  const int64_t oy = y0 > 0 ? min(y0 - 1, M - 1) : 0;
  fw_y[t] = (int32_t)max(count_le(x, N, y[oy], true) - 1, (int64_t)0);
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

finom_status build_plan(finom_plan_s* p, const double* x, const double* y, cudaStream_t s) {
  const int64_t N = p->N, M = p->M, L = N + M;
  p->L = L;
  p->C = (L + kTile - 1) / kTile;
  const int64_t words = (L + 31) / 32;
  // tile-aligned word count so vector loads past L stay inside the allocation
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
  FINOM_CUDA(cudaMemsetAsync(p->tbits, 0, sizeof(uint32_t) * (Lpad / 32), s));
  FINOM_CUDA(cudaMalloc(&p->gap64, sizeof(double) * Lpad));
  FINOM_CUDA(cudaMemsetAsync(p->gap64, 0, sizeof(double) * Lpad, s));
  float* gap32 = nullptr;
  if (p->prec == FINOM_F32_LOG) {
    FINOM_CUDA(cudaMalloc(&gap32, sizeof(float) * Lpad));
    FINOM_CUDA(cudaMemsetAsync(gap32, 0, sizeof(float) * Lpad, s));
    p->gap = gap32;
  } else {
    p->gap = p->gap64;
  }
  FINOM_CUDA(cudaMalloc(&p->tile_x0, sizeof(int32_t) * (p->C + 1)));

  int64_t *posx = nullptr, *posy = nullptr;
  double* z = nullptr;
  uint8_t* type = nullptr;
  FINOM_CUDA(cudaMalloc(&posx, sizeof(int64_t) * N));
  FINOM_CUDA(cudaMalloc(&posy, sizeof(int64_t) * M));
  FINOM_CUDA(cudaMalloc(&z, sizeof(double) * L));
  FINOM_CUDA(cudaMalloc(&type, L));

  k_ranks_x<<<nblk(N, 256), 256, 0, s>>>(p->x, N, p->y, M, p->zeta, posx);
  k_ranks_y<<<nblk(M, 256), 256, 0, s>>>(p->x, N, p->y, M, p->zetaT, posy);
  k_scatter<<<nblk(N, 256), 256, 0, s>>>(p->x, N, posx, z, type, 1);
  k_scatter<<<nblk(M, 256), 256, 0, s>>>(p->y, M, posy, z, type, 0);
  const double inv = 1.0 / (p->eps * std::log(2.0));
  k_gaps_bits<<<nblk(words * 32, 256), 256, 0, s>>>(z, type, L, inv, p->gap64, gap32, p->tbits);
  k_tiles<<<nblk(p->C + 1, 256), 256, 0, s>>>(posx, N, p->C, p->tile_x0);
  FINOM_CUDA(cudaMalloc(&p->fw[0], sizeof(int32_t) * (p->C + 1)));
  FINOM_CUDA(cudaMalloc(&p->fw[1], sizeof(int32_t) * (p->C + 1)));
  k_frame_w<<<nblk(p->C + 1, 256), 256, 0, s>>>(p->x, N, p->y, M, p->zeta, p->tile_x0, p->C, L,
                                                  p->fw[0], p->fw[1]);
  FINOM_CUDA(cudaGetLastError());
  FINOM_CUDA(cudaStreamSynchronize(s));
  cudaFree(posx);
  cudaFree(posy);
  cudaFree(z);
  cudaFree(type);
  p->elems = kElems;
  p->Ce = p->C;
  p->tile_x0e = p->tile_x0;
  return FINOM_OK;
}

finom_status build_tiles_e(finom_plan_s* p, int elems, cudaStream_t s) {
  if (elems != 1 && elems != 2 && elems != 4 && elems != kElems) {
    set_error("points per thread must be 1, 2, 4 or " + std::to_string(kElems));
    return FINOM_EINVAL;
  }
  if (elems == p->elems) return FINOM_OK;
  if (p->tile_x0e && p->tile_x0e != p->tile_x0) cudaFree(p->tile_x0e);
  p->tile_x0e = p->tile_x0;
  p->Ce = p->C;
  p->elems = kElems;
  if (elems == kElems) return FINOM_OK;
  const int64_t tile = (int64_t)elems * kThreads;
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
  if (p->gap && p->gap != p->gap64) cudaFree(p->gap);
  cudaFree(p->gap64);
  if (p->tile_x0e && p->tile_x0e != p->tile_x0) cudaFree(p->tile_x0e);
  cudaFree(p->tile_x0);
  cudaFree(p->fw[0]);
  cudaFree(p->fw[1]);
}

}  // namespace finom
