// Enumeration of the upper block triangle shared by the tile kernels (the
// graph's distance and kernel-value tiles, the CUDA-core chain GEMM and the
// score tiles): tile t of an nb x nb block grid is (bi, bj) with bi <= bj,
// numbered row by row, row bi starting at off(bi) = bi nb - bi (bi - 1) / 2.
#pragma once

#include <cmath>

namespace cdl {

// (bi, bj) of tile t: a float64 estimate from the quadratic, then an exact
// integer correction.
__device__ __forceinline__ void tri_index(long long t, int nb, int& bi, int& bj) {
  double fnb = nb + 0.5;
  int r = (int)floor(fnb - sqrt(fnb * fnb - 2.0 * (double)t));
  if (r < 0) r = 0;
  if (r > nb - 1) r = nb - 1;
  auto off = [nb](long long b) { return b * nb - b * (b - 1) / 2; };
  while (r > 0 && off(r) > t) --r;
  while (r + 1 < nb && off(r + 1) <= t) ++r;
  bi = r;
  bj = r + (int)(t - off(r));
}

// tri_index of the block's own tile, formed once (thread 0: it takes a float64
// square root) and shared; every thread of the block must call it.
__device__ __forceinline__ void block_tri_index(int nb, int& bi, int& bj) {
  __shared__ int tile[2];
  if (threadIdx.x == 0) tri_index(blockIdx.x, nb, tile[0], tile[1]);
  __syncthreads();
  bi = tile[0];
  bj = tile[1];
}

}  // namespace cdl
