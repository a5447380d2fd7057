// Chain-preconditioned Richardson solve of L Z = Y (Alg. 2, EstimateSolution,
// with the k right-hand sides of Alg. 3 processed together as in Sec. 4.1):
//
//   R_0 = Y, Z_0 = 0;  Z_{t+1} = Z_t + P R_t,  R_{t+1} = Y - L Z_{t+1},
//   P R = D^{-1/2} (I + S~_{d-1}) ... (I + S~_0) D^{-1/2} R,
//
// followed after every step by the shift of Z to D-weighted zero column
// means. Starting from zero this is the paper's y_{t+1} = y_t - P2 y_t + chi
// with chi = P1 b and P2 = P1 L. The paper fixes the step count q; here the
// loop also stops once ||R||_F <= rel_tol ||Y||_F.
//
// Residual. The first step forms R = Y - D Z + A Z in full, to float64-class
// accuracy: on tensor-core chains A Z comes from exact bf16 slices of A and
// Z on the tensor cores with integer accumulation (k_tc_resid), on the
// CUDA-core chains from float-float products and sums on the float32 pipes
// (float64 runs at about 1/72 of the float32 rate on this GPU). Later steps
// update it recursively, R -= D dZ - A dZ, on the tensor cores (bf16 hi + lo
// operands) or in float32; each such update adds a bounded error (1e-5 of
// the residual before it), summed as a drift bound. A recursive residual
// that stops falling (less than halved) is formed again in full, and one
// that meets the tolerance is certified by a full residual before the solve
// stops, unless its drift bound is already below a tenth of the tolerance.
// CDL_SOLVE_FULL_RESIDUAL forms it in full on every step.
//
// Tensor-core chains with k > 128 right-hand sides solve them as
// independent column blocks of at most 128 (chain_solve at the end).
#include <cuda_bf16.h>

#include <cmath>
#include <string>
#include <vector>

#include "ff.cuh"
#include "internal.h"

namespace cdl {
namespace {

constexpr int RED_THREADS = 256;

// per-block partial sums of squares (deterministic order)
__global__ void __launch_bounds__(RED_THREADS) k_sumsq(const double* __restrict__ v, size_t count,
                                                        double* __restrict__ part) {
  __shared__ double red[RED_THREADS / 32];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < count;
       i += (size_t)gridDim.x * RED_THREADS) {
    double x = v[i];
    acc = fma(x, x, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_reduce(const double* __restrict__ part, int count, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

template <typename T>
__global__ void k_precond_in(const double* __restrict__ R, const double* __restrict__ rsd, int n,
                             int k, int np, int kp, T* __restrict__ x) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)np * kp) return;
  int i = (int)(idx / kp), r = (int)(idx % kp);
  double v = (i < n && r < k) ? R[(size_t)i * k + r] * rsd[i] : 0.0;
  x[idx] = (T)v;
}

// Z += dZ with dZ = D^{-1/2} x; dZ is also kept in float32 (npad x kp, zero
// padded) for the recursive residual update.
template <typename T>
__global__ void k_precond_out(const T* __restrict__ x, const double* __restrict__ rsd, int n, int k,
                              int np, int kp, double* __restrict__ Z, float* __restrict__ dZ) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)np * kp) return;
  int i = (int)(idx / kp), r = (int)(idx % kp);
  float dzf = 0.f;
  if (i < n && r < k) {
    const double dz = (double)x[idx] * rsd[i];
    Z[(size_t)i * k + r] += dz;
    dzf = (float)dz;
  }
  dZ[idx] = dzf;
}

// x[i][r] += sum_s part[s][i][r] (CUDA-core chains)
template <typename T>
__global__ void k_update_simt(T* __restrict__ x, const T* __restrict__ part, int splits, size_t elems) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= elems) return;
  T acc = x[idx];
  for (int s = 0; s < splits; ++s) acc += part[(size_t)s * elems + idx];
  x[idx] = acc;
}

// bf16 chains: x[i][r] += sum_s (part[s][i][r] + part[s][i][kp + r]) (hi and
// lo halves of the right-hand side), then the tensor-core operand
// xop[r][i] = bf16(x[i][r]), xop[kp + r][i] = bf16(x[i][r] - hi). 32 x 32 tiles.
__global__ void __launch_bounds__(256) k_update_bf16(float* __restrict__ x, const float* __restrict__ part,
                                                      int splits, int np, int kp,
                                                      __nv_bfloat16* __restrict__ xop, int accumulate) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int a = ty; a < 32; a += 8) {
    const int i = i0 + a, r = r0 + tx;
    float v = 0.f;
    if (i < np && r < kp) {
      v = x[(size_t)i * kp + r];
      if (accumulate) {
        for (int s = 0; s < splits; ++s) {
          const float* P = part + ((size_t)s * np + i) * (2 * kp);
          v += P[r] + P[kp + r];
        }
        x[(size_t)i * kp + r] = v;
      }
    }
    tile[a][tx] = v;
  }
  __syncthreads();
  for (int a = ty; a < 32; a += 8) {
    const int r = r0 + a, i = i0 + tx;
    if (r < kp && i < np) {
      const float v = tile[tx][a];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      xop[(size_t)r * np + i] = hi;
      xop[(size_t)(kp + r) * np + i] = lo;
    }
  }
}

// Column sums s_r = sum_i D_i Z[i][r] in fixed-order per-block partials.
__global__ void __launch_bounds__(256) k_colsum_dz(const double* __restrict__ Z, const double* __restrict__ D,
                                                    int n, int k, int rows_per_block, double* __restrict__ part) {
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= k) return;
  const int i0 = blockIdx.x * rows_per_block, i1 = min(n, i0 + rows_per_block);
  double acc = 0.0;
  for (int i = i0; i < i1; ++i) acc = fma(D[i], Z[(size_t)i * k + r], acc);
  part[(size_t)blockIdx.x * k + r] = acc;
}

// shift[r] = (sum of the column's partial sums, in order) / vol, once per column.
__global__ void k_center_shift(const double* __restrict__ part, int nparts, int k, const double* __restrict__ vol,
                               double* __restrict__ shift) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += part[(size_t)p * k + r];
  shift[r] = s / *vol;
}

__global__ void k_center(double* __restrict__ Z, const double* __restrict__ shift, int n, int k) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * k) return;
  Z[idx] -= shift[idx % k];
}

// Z (float64) -> float hi + lo pair for the float-float residual.
__global__ void k_split(const double* __restrict__ Z, size_t count, float* __restrict__ hi,
                        float* __restrict__ lo) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const double z = Z[idx];
  const float h = (float)z;
  hi[idx] = h;
  lo[idx] = (float)(z - (double)h);
}

// Float-float accumulate of (ah + al)(zh + zl) into (s, c): the product's
// rounding error is recovered exactly by fma, the sum's by TwoSum; the
// al * zl term (below 2^-48 relative) is dropped.
__device__ __forceinline__ void ff_mac(float ah, float al, float zh, float zl, float& s, float& c) {
  const float p = __fmul_rn(ah, zh);
  float e = __fmaf_rn(ah, zh, -p);
  e = __fmaf_rn(ah, zl, e);
  e = __fmaf_rn(al, zh, e);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

constexpr int RB_M = 64, RB_N = 64, RB_K = 16;

// R = Y - D o Z + A Z for a TM-row x TN-column tile (64 x 64, or 128 x 32
// for narrow right-hand sides), 4 x 4 float-float accumulators per thread; A
// and Z arrive as float hi + lo planes. Per-block sum of R^2.
template <int TM, int TN>
__device__ __forceinline__ double residual_tile(const float* __restrict__ Ahi, const float* __restrict__ Alo,
                                                const float* __restrict__ Zh, const float* __restrict__ Zl,
                                                const double* __restrict__ Z, const double* __restrict__ Y,
                                                const double* __restrict__ D, int n, int k,
                                                double* __restrict__ R, int i0, int c0) {
  static_assert((TM / 4) * (TN / 4) == 256, "256 threads, 4 x 4 outputs each");
  __shared__ __align__(16) float Ah[RB_K][TM + 4], Al[RB_K][TM + 4];
  __shared__ __align__(16) float Bh[RB_K][TN], Bl[RB_K][TN];
  __shared__ double red[8];
  const int tid = threadIdx.x, tx = tid % (TN / 4), ty = tid / (TN / 4);
  float sh[4][4], sc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) sh[a][b] = sc[a][b] = 0.f;
  for (int j0 = 0; j0 < n; j0 += RB_K) {
#pragma unroll
    for (int e = 0; e < (TM * RB_K) / 256; ++e) {
      const int idx = tid + e * 256;
      const int ii = idx / RB_K, jj = idx % RB_K;
      const int i = i0 + ii, j = j0 + jj;
      const bool ok = i < n && j < n;
      const size_t o = (size_t)i * n + j;
      Ah[jj][ii] = ok ? Ahi[o] : 0.f;
      Al[jj][ii] = ok ? Alo[o] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < (TN * RB_K) / 256; ++e) {
      const int idx = tid + e * 256;
      const int jj = idx / TN, cc = idx % TN;
      const int j = j0 + jj, c = c0 + cc;
      const bool ok = j < n && c < k;
      Bh[jj][cc] = ok ? Zh[(size_t)j * k + c] : 0.f;
      Bl[jj][cc] = ok ? Zl[(size_t)j * k + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < RB_K; ++jj) {
      const float4 ah = *reinterpret_cast<const float4*>(&Ah[jj][ty * 4]);
      const float4 al = *reinterpret_cast<const float4*>(&Al[jj][ty * 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bh[jj][tx * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bl[jj][tx * 4]);
      const float avh[4] = {ah.x, ah.y, ah.z, ah.w}, avl[4] = {al.x, al.y, al.z, al.w};
      const float bvh[4] = {bh.x, bh.y, bh.z, bh.w}, bvl[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ff_mac(avh[a], avl[a], bvh[b], bvl[b], sh[a][b], sc[a][b]);
    }
    __syncthreads();
    // renormalise (s, c) so that the compensation stays below ulp(s): its own
    // rounding errors then stay at 2^-48 of the sum per step
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const ff r = two_sum(sh[a][b], sc[a][b]);
        sh[a][b] = r.hi;
        sc[a][b] = r.lo;
      }
  }
  double sq = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
    if (i >= n) continue;
    const double di = D[i];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= k) continue;
      const size_t o = (size_t)i * k + c;
      const double az = (double)sh[a][b] + (double)sc[a][b];
      const double r = (Y[o] - di * Z[o]) + az;
      R[o] = r;
      sq = fma(r, r, sq);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((tid & 31) == 0) red[tid >> 5] = sq;
  __syncthreads();
  double t = 0.0;
  if (tid == 0)
    for (int w = 0; w < 8; ++w) t += red[w];
  return t;   // valid in thread 0
}

__global__ void __launch_bounds__(256) k_residual(const float* __restrict__ Ahi, const float* __restrict__ Alo,
                                                   const float* __restrict__ Zh, const float* __restrict__ Zl,
                                                   const double* __restrict__ Z, const double* __restrict__ Y,
                                                   const double* __restrict__ D, int n, int k,
                                                   double* __restrict__ R, double* __restrict__ part) {
  const double t = residual_tile<RB_M, RB_N>(Ahi, Alo, Zh, Zl, Z, Y, D, n, k, R, blockIdx.x * RB_M,
                                             blockIdx.y * RB_N);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Recursive residual update R -= D o dZ - A dZ for a 128-row x 128-column
// tile (8 x 8 outputs per thread), A dZ accumulated in float32; per-block sum of
// the new R^2. The update is small (|dZ| shrinks with the residual), so its
// float32 error, about 1e-7 of ||L dZ||, stays far below the float-float
// residual it corrects.
constexpr int RU_M = 128, RU_N = 128, RU_K = 16;
__global__ void __launch_bounds__(256) k_residual_update(const double* __restrict__ A, const float* __restrict__ dZ,
                                                          const double* __restrict__ D, int n, int k, int kp,
                                                          double* __restrict__ R, double* __restrict__ part) {
  __shared__ __align__(16) float As[RU_K][RU_M + 4];
  __shared__ __align__(16) float Bs[RU_K][RU_N];
  __shared__ double red[8];
  const int i0 = blockIdx.x * RU_M, c0 = blockIdx.y * RU_N;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int j0 = 0; j0 < n; j0 += RU_K) {
#pragma unroll
    for (int e = 0; e < (RU_M * RU_K) / 256; ++e) {
      const int idx = tid + e * 256;
      const int ii = idx / RU_K, jj = idx % RU_K;
      const int i = i0 + ii, j = j0 + jj;
      As[jj][ii] = (i < n && j < n) ? __double2float_rn(A[(size_t)i * n + j]) : 0.f;
    }
#pragma unroll
    for (int e = 0; e < (RU_N * RU_K) / 256; ++e) {
      const int idx = tid + e * 256;
      const int jj = idx / RU_N, cc = idx % RU_N;
      const int j = j0 + jj, c = c0 + cc;
      Bs[jj][cc] = (j < n && c < k) ? dZ[(size_t)j * kp + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < RU_K; ++jj) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[jj][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[jj][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[jj][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[jj][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = __fmaf_rn(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  double sq = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
    if (i >= n) continue;
    const double di = D[i];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int c = c0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4);
      if (c >= k) continue;
      const size_t o = (size_t)i * k + c;
      const double r = R[o] - (di * (double)dZ[(size_t)i * kp + c] - (double)acc[a][b]);
      R[o] = r;
      sq = fma(r, r, sq);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((tid & 31) == 0) red[tid >> 5] = sq;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// The value of dZ the tensor-core products see: its bf16 hi + lo split.
// The diagonal term D o dZ uses the same value, so that the update applies
// one operator to one vector: were D o dZ taken at full float precision, the
// common rounding of a column's constant part (which A, close to a multiple
// of the all-ones matrix, sums n times) would leave a residual along D 1
// that the deflated preconditioner cannot see, and the refinement would stall.
__device__ __forceinline__ float bf16_pair_value(float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  return __bfloat162float(hi) + __bfloat162float(lo);
}

// Tensor-core residual update, second half: the products A_hi [dZ_hi|dZ_lo]
// and A_lo [dZ_hi|dZ_lo] arrive as float32 split-K partials (bf16 operands:
// about 16 significant bits of A and of dZ); R -= D o dZ - (sum of the four
// products) with dZ as the products see it; per-block sums of the new R^2.
__global__ void __launch_bounds__(256) k_residual_update_tc(const float* __restrict__ pa, const float* __restrict__ pb,
                                                             int splits, int np, const float* __restrict__ dZ,
                                                             const double* __restrict__ D, int n, int k, int kp,
                                                             double* __restrict__ R, double* __restrict__ part) {
  __shared__ double red[8];
  double sq = 0.0;
  const size_t total = (size_t)n * k;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k), c = (int)(idx % k);
    double az = 0.0;
    for (int s = 0; s < splits; ++s) {
      const size_t o = ((size_t)s * np + i) * (2 * kp);
      az += (double)pa[o + c] + (double)pa[o + kp + c] + (double)pb[o + c] + (double)pb[o + kp + c];
    }
    const double r = R[idx] - (D[i] * (double)bf16_pair_value(dZ[(size_t)i * kp + c]) - az);
    R[idx] = r;
    sq = fma(r, r, sq);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}


// ---- exact-slice residual (tensor chains): Z / c_r in six bf16 slices,
// c_r the power of two just above column r's largest |Z|.
__global__ void k_zcolmax(const double* __restrict__ Z, size_t count, int k, unsigned long long* __restrict__ mbits) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x)
    atomicMax(mbits + idx % k, (unsigned long long)__double_as_longlong(fabs(Z[idx])));
}

__device__ __forceinline__ double pow2_above(unsigned long long bits) {
  if (bits == 0) return 1.0;
  const int e = (int)((bits >> 52) & 0x7FF);
  return ldexp(1.0, e - 1022);
}

// planes S[t][rl][j] (t = 0..5, rl < kg, j < npad) for columns c0 + rl.
__global__ void __launch_bounds__(256) k_zslice(const double* __restrict__ Z, int n, int k, int np, int c0, int kg,
                                                 const unsigned long long* __restrict__ mbits,
                                                 __nv_bfloat16* __restrict__ S, double* __restrict__ cs) {
  const size_t plane = (size_t)kg * np;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane; idx += (size_t)gridDim.x * blockDim.x) {
    const int rl = (int)(idx / np), j = (int)(idx % np);
    const int r = c0 + rl;
    long long N = 0;
    if (r < k) {
      const double c = pow2_above(mbits[r]);
      if (j == 0) cs[r] = c;
      if (j < n) N = llrint(Z[(size_t)j * k + r] / c * 0x1p48);   // |Z / c| < 1, division by a power of two is exact
    }
#pragma unroll
    for (int t = 1; t <= 6; ++t) {
      const int sh = 48 - 8 * t;
      long long d = N;
      if (sh > 0) d = (N + (1LL << (sh - 1))) >> sh;
      N -= d << sh;
      S[(size_t)(t - 1) * plane + idx] = __float2bfloat16_rn(ldexpf((float)d, -8 * t));
    }
  }
}

// R = (Y - D o Z) + (2^s c_r) G (G from the column groups of at most 128,
// each the sum of its RESID_PAIRS slice-pair planes; 2^s = a_scale[0], the
// scale of A's slices), and per-block sums of R^2.
__global__ void __launch_bounds__(256) k_resid_combine(const double* __restrict__ Y, const double* __restrict__ Z,
                                                        const double* __restrict__ D, int n, int k, int np,
                                                        const double* __restrict__ G, const double* __restrict__ cs,
                                                        const double* __restrict__ a_scale,
                                                        double* __restrict__ R, double* __restrict__ part) {
  __shared__ double red[8];
  const double as = a_scale[0];
  double sq = 0.0;
  const size_t total = (size_t)n * k;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k), r = (int)(idx % k);
    const int g = r / 128, rl = r % 128;
    const int kg = min(128, ((k - g * 128) + 31) / 32 * 32);
    const double* Gg = G + (size_t)g * RESID_PAIRS * np * 128 + (size_t)i * kg + rl;
    double sum = 0.0;
    for (int pr = 0; pr < RESID_PAIRS; ++pr) sum += Gg[(size_t)pr * np * kg];   // the slice pairs in order
    const double az = (cs[r] * as) * sum;   // powers of two: exact
    const double v = (Y[idx] - D[i] * Z[idx]) + az;
    R[idx] = v;
    sq = fma(v, v, sq);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- batched form
// The kernels below run one step of the refinement for every graph of a
// batch in one launch; a block finds its graph and block index in a tile
// table and returns at once when its graph's command does not include the
// step (converged graphs cost one load per block).

__device__ __forceinline__ void tdec(uint32_t t, int& g, int& b) {
  g = (int)(t & 0xFFFu);
  b = (int)(t >> 12);
}

// sum over a 256-thread block in a fixed order (result in thread 0)
__device__ __forceinline__ double block_sum256(double v) {
  __shared__ double sh[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) t += sh[w];
  return t;
}

// R = Y, Z = 0, and per-block sums of Y^2.
__global__ void __launch_bounds__(256) k_b_start(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                  int k) {
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  const BGraph& G = gs[g];
  const size_t idx = (size_t)b * 256 + threadIdx.x;
  double y2 = 0.0;
  if (idx < (size_t)G.n * k) {
    const double y = G.Y[idx];
    G.R[idx] = y;
    G.Z[idx] = 0.0;
    y2 = y * y;
  }
  const double t = block_sum256(y2);
  if (threadIdx.x == 0) G.red[b] = t;
}

// ||Y||^2 per graph and the first command (a step with a full residual).
__global__ void __launch_bounds__(256) k_b_begin(const BGraph* __restrict__ gs, BState* __restrict__ st) {
  const BGraph& G = gs[blockIdx.x];
  double acc = 0.0;
  for (int b = threadIdx.x; b < G.elem_blocks; b += 256) acc += G.red[b];
  const double yy = block_sum256(acc);
  if (threadIdx.x == 0) {
    BState& s = st[blockIdx.x];
    s.yy = yy;
    s.iters = 0;
    s.exact = 1;
    s.drift = 0.0;
    s.rel = yy > 0.0 ? 1.0 : 0.0;
    for (int h = 0; h < 64; ++h) s.hist[h] = 0.0;
    s.cmd = yy > 0.0 ? (CMD_STEP | CMD_FULL) : 0;
  }
}

// bf16 hi/lo transposed operand of a 32-row block: op[r][i], op[kp + r][i].
__device__ __forceinline__ void write_op_tile(float (*tile)[33], int i0, int r0, int kp, int np,
                                              __nv_bfloat16* __restrict__ op) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int a = ty; a < 32; a += 8) {
    const int r = r0 + a, i = i0 + tx;
    if (r < kp) {
      const float v = tile[tx][a];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      op[(size_t)r * np + i] = hi;
      op[(size_t)(kp + r) * np + i] = lo;
    }
  }
}

// x = D^{-1/2} R (float, zero padded) and its bf16 operand.
__global__ void __launch_bounds__(256) k_b_precond_in(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                       const BState* __restrict__ st, int k, int kp) {
  __shared__ float tile[32][33];
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_STEP)) return;
  const BGraph& G = gs[g];
  const int i0 = b * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r0 = 0; r0 < kp; r0 += 32) {
    for (int a = ty; a < 32; a += 8) {
      const int i = i0 + a, r = r0 + tx;
      const float v = (i < G.n && r < k) ? (float)(G.R[(size_t)i * k + r] * G.rsd[i]) : 0.f;
      if (r < kp) G.x[(size_t)i * kp + r] = v;
      tile[a][tx] = v;
    }
    __syncthreads();
    write_op_tile(tile, i0, r0, kp, G.np, static_cast<__nv_bfloat16*>(G.xop));
    __syncthreads();
  }
}

// x += (I + S~) contribution of one level: x += part_hi + part_lo; new operand.
__global__ void __launch_bounds__(256) k_b_update(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                   const BState* __restrict__ st, int kp) {
  __shared__ float tile[32][33];
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_STEP)) return;
  const BGraph& G = gs[g];
  const int i0 = b * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r0 = 0; r0 < kp; r0 += 32) {
    for (int a = ty; a < 32; a += 8) {
      const int i = i0 + a, r = r0 + tx;
      float v = 0.f;
      if (r < kp) {
        const float* P = G.part + (size_t)i * (2 * kp);
        v = G.x[(size_t)i * kp + r];
        v += P[r] + P[kp + r];
        G.x[(size_t)i * kp + r] = v;
      }
      tile[a][tx] = v;
    }
    __syncthreads();
    write_op_tile(tile, i0, r0, kp, G.np, static_cast<__nv_bfloat16*>(G.xop));
    __syncthreads();
  }
}

// Z += dZ = D^{-1/2} x; dZ kept in float (and as a bf16 operand when the
// residual is updated recursively).
__global__ void __launch_bounds__(256) k_b_precond_out(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                        const BState* __restrict__ st, int k, int kp) {
  __shared__ float tile[32][33];
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  const int cmd = st[g].cmd;
  if (!(cmd & CMD_STEP)) return;
  const BGraph& G = gs[g];
  const int i0 = b * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r0 = 0; r0 < kp; r0 += 32) {
    for (int a = ty; a < 32; a += 8) {
      const int i = i0 + a, r = r0 + tx;
      float dzf = 0.f;
      if (i < G.n && r < k) {
        const double dz = (double)G.x[(size_t)i * kp + r] * G.rsd[i];
        G.Z[(size_t)i * k + r] += dz;
        dzf = (float)dz;
      }
      if (r < kp) G.dz[(size_t)i * kp + r] = dzf;
      tile[a][tx] = dzf;
    }
    __syncthreads();
    if (cmd & CMD_RECUR) write_op_tile(tile, i0, r0, kp, G.np, static_cast<__nv_bfloat16*>(G.dzop));
    __syncthreads();
  }
}

// Column sums of D o Z over 256-row chunks (fixed order).
__global__ void __launch_bounds__(256) k_b_colsum(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                   const BState* __restrict__ st, int k) {
  __shared__ double sh[8][33];
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_STEP)) return;
  const BGraph& G = gs[g];
  const int i0 = b * 256, i1 = min(G.n, i0 + 256);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r0 = 0; r0 < k; r0 += 32) {
    const int r = r0 + tx;
    double acc = 0.0;
    if (r < k)
      for (int i = i0 + ty; i < i1; i += 8) acc = fma(G.D[i], G.Z[(size_t)i * k + r], acc);
    sh[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && r < k) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += sh[q][tx];
      G.cs[(size_t)b * k + r] = t;
    }
    __syncthreads();
  }
}

// D-weighted centring: Z -= (sum_i D_i Z_i) / vol.
__global__ void __launch_bounds__(256) k_b_center(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                   const BState* __restrict__ st, int k) {
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_STEP)) return;
  const BGraph& G = gs[g];
  const size_t idx = (size_t)b * 256 + threadIdx.x;
  if (idx >= (size_t)G.n * k) return;
  const int r = (int)(idx % k);
  const int nparts = (G.n + 255) / 256;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += G.cs[(size_t)q * k + r];
  G.Z[idx] -= s / *G.vol;
}

// Full residual of the graphs due one (the exact-slice form of the single
// graph path, Sec. 5): max |Z| per column ...
__global__ void __launch_bounds__(256) k_b_zcolmax(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                    const BState* __restrict__ st, int k) {
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_FULL)) return;
  const BGraph& G = gs[g];
  const size_t idx = (size_t)b * 256 + threadIdx.x;
  if (idx >= (size_t)G.n * k) return;
  atomicMax(G.zmax + idx % k, (unsigned long long)__double_as_longlong(fabs(G.Z[idx])));
}

// ... the six exact slices of Z / c, transposed (kg x npad), and c per column ...
__global__ void __launch_bounds__(256) k_b_zslice(const uint32_t* __restrict__ tiles, const BGraph* __restrict__ gs,
                                                   const BState* __restrict__ st, int k) {
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_FULL)) return;
  const BGraph& G = gs[g];
  const size_t plane = (size_t)G.kg * G.np;
  const size_t idx = (size_t)b * 256 + threadIdx.x;
  if (idx >= plane) return;
  const int r = (int)(idx / G.np), j = (int)(idx % G.np);
  long long N = 0;
  if (r < k) {
    const double c = pow2_above(G.zmax[r]);
    if (j == 0) G.zc[r] = c;
    if (j < G.n) N = llrint(G.Z[(size_t)j * k + r] / c * 0x1p48);   // |Z / c| < 1; the division is exact
  }
  __nv_bfloat16* S = static_cast<__nv_bfloat16*>(G.zs);
#pragma unroll
  for (int t = 1; t <= 6; ++t) {
    const int sh = 48 - 8 * t;
    long long d = N;
    if (sh > 0) d = (N + (1LL << (sh - 1))) >> sh;
    N -= d << sh;
    S[(size_t)(t - 1) * plane + idx] = __float2bfloat16_rn(ldexpf((float)d, -8 * t));
  }
}

// ... and, after the slice products (resid_tc_grouped), R = Y - D o Z + c A Z
// with A Z the sum of the RESID_PAIRS planes in pair order; per-block sums of
// R^2 (the kernel graphs' slices carry scale 2^0).
__global__ void __launch_bounds__(256) k_b_resid_combine(const uint32_t* __restrict__ tiles,
                                                          const BGraph* __restrict__ gs,
                                                          const BState* __restrict__ st, int k) {
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_FULL)) return;
  const BGraph& G = gs[g];
  const size_t idx = (size_t)b * 256 + threadIdx.x;
  double sq = 0.0;
  if (idx < (size_t)G.n * k) {
    const int i = (int)(idx / k), r = (int)(idx % k);
    const size_t pl = (size_t)G.np * G.kg;
    const double* Gg = G.Gp + (size_t)i * G.kg + r;
    double sum = 0.0;
    for (int pr = 0; pr < RESID_PAIRS; ++pr) sum += Gg[(size_t)pr * pl];   // the slice pairs in order
    const double v = (G.Y[idx] - G.D[i] * G.Z[idx]) + G.zc[r] * sum;   // a power of two: exact
    G.R[idx] = v;
    sq = v * v;
  }
  const double t = block_sum256(sq);
  if (threadIdx.x == 0) G.red[b] = t;
}

// Recursive update R -= D o dZ - A dZ from the tensor-core products.
__global__ void __launch_bounds__(256) k_b_residual_update(const uint32_t* __restrict__ tiles,
                                                            const BGraph* __restrict__ gs,
                                                            const BState* __restrict__ st, int k, int kp) {
  int g, b;
  tdec(tiles[blockIdx.x], g, b);
  if (!(st[g].cmd & CMD_RECUR)) return;
  const BGraph& G = gs[g];
  const size_t idx = (size_t)b * 256 + threadIdx.x;
  double sq = 0.0;
  if (idx < (size_t)G.n * k) {
    const int i = (int)(idx / k), c = (int)(idx % k);
    const size_t o = (size_t)i * (2 * kp);
    double az = 0.0;
    az += (double)G.part[o + c] + (double)G.part[o + kp + c] + (double)G.part2[o + c] + (double)G.part2[o + kp + c];
    const double r = G.R[idx] - (G.D[i] * (double)bf16_pair_value(G.dz[(size_t)i * kp + c]) - az);
    G.R[idx] = r;
    sq = r * r;
  }
  const double t = block_sum256(sq);
  if (threadIdx.x == 0) G.red[b] = t;
}

// Residual norm of each graph and its next command: stop when the residual is
// certified below the tolerance, or at the iteration cap or on divergence;
// certify a recursively updated residual with a full one before stopping.
__global__ void __launch_bounds__(256) k_b_decide(const BGraph* __restrict__ gs, BState* __restrict__ st,
                                                   double tol, int max_iter, int always_full,
                                                   int* __restrict__ active) {
  const int g = blockIdx.x;
  const int cmd = st[g].cmd;
  if (cmd == 0) return;
  const BGraph& G = gs[g];
  const int cnt = (cmd & CMD_FULL) ? G.res_tiles : G.elem_blocks;
  double acc = 0.0;
  for (int b = threadIdx.x; b < cnt; b += 256) acc += G.red[b];
  const double rr = block_sum256(acc);
  if (threadIdx.x != 0) return;
  BState& s = st[g];
  if (cmd & CMD_STEP) {
    s.iters += 1;
    if (cmd & CMD_RECUR) {
      s.drift += 1e-5 * s.rel;   // error of the L dZ product, |L dZ| ~ |R| before the step
      s.exact = 0;
    }
  }
  if (cmd & CMD_FULL) {
    s.exact = 1;
    s.drift = 0.0;
  }
  const double rel = sqrt(rr / s.yy);
  const double prev = s.rel;
  s.rel = rel;
  if (s.iters >= 1 && s.iters <= 64) s.hist[s.iters - 1] = rel;
  int next;
  if (!s.exact && rel > 0.5 * prev) {
    next = CMD_FULL;   // a recursive residual that stops falling: form it in full
  } else if (tol > 0 && rel <= tol) {
    next = (!s.exact && rel + s.drift > 0.1 * tol) ? CMD_FULL : 0;
  } else if (s.iters >= max_iter || !(rel <= 1e6)) {
    next = 0;
  } else {
    next = CMD_STEP | (always_full ? CMD_FULL : CMD_RECUR);
  }
  s.cmd = next;
  if (next) atomicAdd(active, 1);
}

int largest_divisor_at_most(int total, int target) {
  int best = 1;
  for (int s = 1; s <= total && s <= target; ++s)
    if (total % s == 0) best = s;
  return best;
}

inline unsigned blocks_for(size_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

}  // namespace

namespace {

// One block of at most 128 right-hand sides (any number for CUDA-core
// chains) of the Richardson refinement, with its own residual, iterate,
// operand buffers and stopping state; chain_solve steps every block together
// so that each chain level is applied to all of them while it is loaded.
struct SolveBlock {
  cdl_ctx* ctx = nullptr;
  const cdl_chain* ch = nullptr;
  const double* A = nullptr;
  const double* Y = nullptr;
  double* Z = nullptr;
  cdl_solve_stats* stats = nullptr;
  cudaStream_t st = nullptr;
  int n = 0, np = 0, k = 0, kp = 0, splits = 1;
  bool bf16 = false;
  size_t xe = 4, nk = 0;
  int res_gx = 0, res_gy = 0, upd_gx = 0, upd_gy = 0, cs_rows = 256, cs_parts = 0;
  void *vR = nullptr, *vx = nullptr, *vxop = nullptr, *vpart = nullptr, *vred = nullptr, *vscal = nullptr;
  void *vzh = nullptr, *vzl = nullptr, *vcs = nullptr, *vdz = nullptr, *vpart2 = nullptr, *vdzop = nullptr;
  double *R = nullptr, *red = nullptr, *scal = nullptr;
  double yy = 0.0, rel = 1.0, drift = 0.0;
  int iters = 0, nparts = 0;
  bool exact_r = true;   // R was last formed in full (not recursively)
  bool done = false;

  int ws(const char* name, int idx, size_t bytes, void** out) {
    if (idx == 0) return ws_get(ctx, name, bytes, out);
    const std::string nm = std::string(name) + "#" + std::to_string(idx);
    return ws_get(ctx, nm.c_str(), bytes, out);
  }

  // workspace (block idx > 0 under its own names), ||Y||^2, Z = 0, R = Y
  int init(int idx) {
    st = ctx->stream;
    n = (int)ch->n;
    np = (int)ch->npad;
    kp = (int)round_up(k, 16);   // tensor-core N = 2 kp: multiple of 32
    bf16 = ch->dtype == CDL_BF16 || ch->dtype == CDL_FP8E4M3 || ch->dtype == CDL_FP8E4M3_T128;   // tensor-core apply
    xe = ch->dtype == CDL_F64 ? 8 : 4;
    const int kblocks = np / 64;
    if (bf16) {
      // split-K of the persistent apply (one CTA per SM over np / 128 row tiles x
      // splits): the fewest splits (a divisor of the K blocks, at most 16) whose
      // tiles fill the last round of CTAs to 95 %, else the best filling
      const int mb = np / 128, sm = ctx->sm_count;
      splits = 1;
      double best = 0.0;
      for (int sp = 1; sp <= 16 && sp <= kblocks; ++sp) {
        if (kblocks % sp) continue;
        const long long tl = (long long)mb * sp;
        const double fill = (double)tl / (double)(((tl + sm - 1) / sm) * sm);
        if (fill > best + 1e-9) {
          best = fill;
          splits = sp;
        }
        if (fill >= 0.95) break;
      }
    } else {
      const int bm = ch->dtype == CDL_F32 ? 128 : 64;
      const int cols = (kp + 63) / 64;
      const int target = std::max(1, (8 * ctx->sm_count) / ((np / bm) * cols));
      splits = largest_divisor_at_most(np / 8, std::min(target, 16));
    }
    const size_t part_cols = bf16 ? 2 * (size_t)kp : (size_t)kp;
    res_gx = (n + RB_M - 1) / RB_M;
    res_gy = (k + RB_N - 1) / RB_N;
    upd_gx = (n + RU_M - 1) / RU_M;
    upd_gy = (k + RU_N - 1) / RU_N;
    const int nred = std::max(res_gx * res_gy, std::max(1024, ctx->sm_count * 4));
    cs_parts = (n + cs_rows - 1) / cs_rows;
    CDL_TRY(ws("solve.R", idx, (size_t)n * k * 8, &vR));
    CDL_TRY(ws("solve.x", idx, (size_t)np * kp * xe, &vx));
    if (bf16) CDL_TRY(ws("solve.xop", idx, 2 * (size_t)kp * np * 2, &vxop));
    CDL_TRY(ws("solve.part", idx, (size_t)splits * np * part_cols * xe, &vpart));
    CDL_TRY(ws("solve.red", idx, (size_t)nred * 8, &vred));
    CDL_TRY(ws("solve.scal", idx, 64, &vscal));
    CDL_TRY(ws("solve.zh", idx, (size_t)n * k * 4, &vzh));
    CDL_TRY(ws("solve.zl", idx, (size_t)n * k * 4, &vzl));
    CDL_TRY(ws("solve.colsum", idx, (size_t)(cs_parts + 1) * k * 8, &vcs));   // partial sums, then the shift
    CDL_TRY(ws("solve.dz", idx, (size_t)np * kp * 4, &vdz));
    if (bf16) {
      CDL_TRY(ws("solve.part2", idx, (size_t)splits * np * part_cols * xe, &vpart2));
      CDL_TRY(ws("solve.dzop", idx, 2 * (size_t)kp * np * 2, &vdzop));
    }
    R = static_cast<double*>(vR);
    red = static_cast<double*>(vred);
    scal = static_cast<double*>(vscal);
    nk = (size_t)n * k;
    nparts = res_gx * res_gy;   // per-block partial sums of R^2 written by the last residual kernel
    {
      const int nb = (int)std::min<size_t>(1024, (nk + RED_THREADS - 1) / RED_THREADS);
      {
        Launch L(ctx, CDL_KC_MISC, 0);
        k_sumsq<<<nb, RED_THREADS, 0, st>>>(Y, nk, red);
        CDL_TRY(L.done());
      }
      {
        Launch L(ctx, CDL_KC_MISC, 0);
        k_reduce<<<1, 1024, 0, st>>>(red, nb, scal);
        CDL_TRY(L.done());
      }
      CDL_CUDA_TRY(cudaMemcpyAsync(&yy, scal, 8, cudaMemcpyDeviceToHost, st));
      CDL_CUDA_TRY(cudaStreamSynchronize(st));
    }
    CDL_CUDA_TRY(cudaMemsetAsync(Z, 0, nk * 8, st));
    CDL_CUDA_TRY(cudaMemcpyAsync(R, Y, nk * 8, cudaMemcpyDeviceToDevice, st));
    if (stats) {
      stats->iters = 0;
      stats->rel_res = yy > 0 ? 1.0 : 0.0;
      for (double& h : stats->history) h = 0.0;
    }
    done = yy == 0.0;
    rel = yy > 0 ? 1.0 : 0.0;
    return CDL_OK;
  }

  // Full residual R = Y - L Z (float64-class).
  int full_residual() {
    if (ch->regen) {
      // A Z of a graph regenerated panel by panel: each panel's transposed
      // exact slices are one K range of A Z (A symmetric), added into G
      const RegenSource& rs = *ch->regen;
      const int ngroups = (k + 127) / 128;
      void *vzs, *vG, *vmb, *vcz;
      CDL_TRY(ws_get(ctx, "solve.zslices", 6 * (size_t)128 * np * 2, &vzs));
      CDL_TRY(ws_get(ctx, "solve.G", (size_t)ngroups * RESID_PAIRS * np * 128 * sizeof(double), &vG));
      CDL_TRY(ws_get(ctx, "solve.zmax", (size_t)k * 8, &vmb));
      CDL_TRY(ws_get(ctx, "solve.zc", (size_t)k * 8, &vcz));
      CDL_CUDA_TRY(cudaMemsetAsync(vmb, 0, (size_t)k * 8, st));
      {
        Launch L(ctx, CDL_KC_MISC, 0);
        k_zcolmax<<<std::min<size_t>(blocks_for(nk, 256), (size_t)ctx->sm_count * 8), 256, 0, st>>>(
            Z, nk, k, static_cast<unsigned long long*>(vmb));
        CDL_TRY(L.done());
      }
      for (int g = 0; g < ngroups; ++g) {
        const int c0 = g * 128;
        const int kg = std::min(128, (k - c0 + 31) / 32 * 32);
        double* Gg = static_cast<double*>(vG) + (size_t)g * RESID_PAIRS * np * 128;
        {
          Launch L(ctx, CDL_KC_MISC, 0);
          k_zslice<<<ctx->sm_count * 4, 256, 0, st>>>(Z, n, k, np, c0, kg,
                                                       static_cast<const unsigned long long*>(vmb),
                                                       static_cast<__nv_bfloat16*>(vzs), static_cast<double*>(vcz));
          CDL_TRY(L.done());
        }
        CDL_CUDA_TRY(cudaMemsetAsync(Gg, 0, (size_t)RESID_PAIRS * np * kg * sizeof(double), st));
        for (int r0 = 0; r0 < n; r0 += rs.P) {
          const int rows = std::min(rs.P, n - r0);
          CDL_TRY(regen_panel(ctx, *rs.g, rs.panel, r0, rows, rs.Dscratch));
          CDL_TRY(panel_slices_t(ctx, rs.panel, n, np, r0, rows, rs.P, rs.slicesT));
          CDL_TRY(resid_tc_panel(ctx, rs.slicesT, np, rs.P, std::min(rs.P, np - r0), r0, vzs, kg, Gg));
        }
      }
      const int nb = std::min(1024, (int)blocks_for(nk, 256));
      Launch L(ctx, CDL_KC_RESIDUAL, 0);
      k_resid_combine<<<nb, 256, 0, st>>>(Y, Z, ch->D, n, k, np, static_cast<const double*>(vG),
                                          static_cast<const double*>(vcz), ch->a_scale, R, red);
      CDL_TRY(L.done());
      nparts = nb;
      return CDL_OK;
    }
    if (ch->aslices) {
      // A Z from exact bf16 slices on the tensor cores, in column groups of <= 128
      const int ngroups = (k + 127) / 128;
      void *vzs, *vG, *vmb, *vcz;
      CDL_TRY(ws_get(ctx, "solve.zslices", 6 * (size_t)128 * np * 2, &vzs));
      CDL_TRY(ws_get(ctx, "solve.G", (size_t)ngroups * RESID_PAIRS * np * 128 * sizeof(double), &vG));
      CDL_TRY(ws_get(ctx, "solve.zmax", (size_t)k * 8, &vmb));
      CDL_TRY(ws_get(ctx, "solve.zc", (size_t)k * 8, &vcz));
      CDL_CUDA_TRY(cudaMemsetAsync(vmb, 0, (size_t)k * 8, st));
      {
        Launch L(ctx, CDL_KC_MISC, 0);
        k_zcolmax<<<std::min<size_t>(blocks_for(nk, 256), (size_t)ctx->sm_count * 8), 256, 0, st>>>(
            Z, nk, k, static_cast<unsigned long long*>(vmb));
        CDL_TRY(L.done());
      }
      for (int g = 0; g < ngroups; ++g) {
        const int c0 = g * 128;
        const int kg = std::min(128, (k - c0 + 31) / 32 * 32);
        {
          Launch L(ctx, CDL_KC_MISC, 0);
          k_zslice<<<ctx->sm_count * 4, 256, 0, st>>>(Z, n, k, np, c0, kg,
                                                       static_cast<const unsigned long long*>(vmb),
                                                       static_cast<__nv_bfloat16*>(vzs), static_cast<double*>(vcz));
          CDL_TRY(L.done());
        }
        CDL_TRY(resid_tc(ctx, ch, vzs, kg, static_cast<double*>(vG) + (size_t)g * RESID_PAIRS * np * 128));
      }
      const int nb = std::min(1024, (int)blocks_for(nk, 256));
      Launch L(ctx, CDL_KC_RESIDUAL, 0);
      k_resid_combine<<<nb, 256, 0, st>>>(Y, Z, ch->D, n, k, np, static_cast<const double*>(vG),
                                          static_cast<const double*>(vcz), ch->a_scale, R, red);
      CDL_TRY(L.done());
      nparts = nb;
      return CDL_OK;
    }
    {
      Launch L(ctx, CDL_KC_MISC, 0);
      k_split<<<blocks_for(nk, 256), 256, 0, st>>>(Z, nk, static_cast<float*>(vzh), static_cast<float*>(vzl));
      CDL_TRY(L.done());
    }
    {
      dim3 g(res_gx, res_gy);
      Launch L(ctx, CDL_KC_RESIDUAL, (double)n * n * k);
      k_residual<<<g, 256, 0, st>>>(ch->ahl, ch->ahl + (size_t)n * n, static_cast<const float*>(vzh),
                                     static_cast<const float*>(vzl), Z, Y, ch->D, n, k, R, red);
      CDL_TRY(L.done());
    }
    nparts = res_gx * res_gy;
    return CDL_OK;
  }

  // Recursive update R -= L dZ in float32.
  int update_residual() {
    if (bf16 && ch->aop) {
      // dZ -> bf16 hi/lo operand, then A_hi and A_lo times it on the tensor cores
      {
        dim3 g((np + 31) / 32, (kp + 31) / 32);
        Launch L(ctx, CDL_KC_MISC, 0);
        k_update_bf16<<<g, 256, 0, st>>>(static_cast<float*>(vdz), nullptr, 0, np, kp,
                                         static_cast<__nv_bfloat16*>(vdzop), 0);
        CDL_TRY(L.done());
      }
      const __nv_bfloat16* ahi = static_cast<const __nv_bfloat16*>(ch->aop);
      CDL_TRY(apply_tc_mat(ctx, ahi, np, vdzop, static_cast<float*>(vpart), kp, splits));
      CDL_TRY(apply_tc_mat(ctx, ahi + (size_t)np * np, np, vdzop, static_cast<float*>(vpart2), kp, splits));
      const int nb = (int)std::min<size_t>((nk + 255) / 256, (size_t)ctx->sm_count * 4);
      Launch L(ctx, CDL_KC_RESIDUAL, 0);
      k_residual_update_tc<<<nb, 256, 0, st>>>(static_cast<const float*>(vpart), static_cast<const float*>(vpart2),
                                               splits, np, static_cast<const float*>(vdz), ch->D, n, k, kp, R, red);
      nparts = nb;
      return L.done();
    }
    dim3 g(upd_gx, upd_gy);
    Launch L(ctx, CDL_KC_RESIDUAL, (double)n * n * k);
    k_residual_update<<<g, 256, 0, st>>>(A, static_cast<const float*>(vdz), ch->D, n, k, kp, R, red);
    nparts = upd_gx * upd_gy;
    return L.done();
  }

  int read_norm() {
    double rr = 0.0;
    {
      Launch L(ctx, CDL_KC_MISC, 0);
      k_reduce<<<1, 1024, 0, st>>>(red, nparts, scal + 1);
      CDL_TRY(L.done());
    }
    CDL_CUDA_TRY(cudaMemcpyAsync(&rr, scal + 1, 8, cudaMemcpyDeviceToHost, st));
    CDL_CUDA_TRY(cudaStreamSynchronize(st));
    rel = std::sqrt(rr / yy);
    return CDL_OK;
  }

  // Before a step: stop when the residual is certified below the tolerance
  // (a recursively updated one is formed in full first unless its drift
  // bound is below a tenth of it), at the iteration cap, or on divergence.
  int pre_step(const cdl_solve_opts* opts) {
    while (true) {
      if (opts->rel_tol > 0 && rel <= opts->rel_tol) {
        if (!exact_r && rel + drift > 0.1 * opts->rel_tol) {
          CDL_TRY(full_residual());
          CDL_TRY(read_norm());
          exact_r = true;
          drift = 0.0;
          if (stats && iters >= 1 && iters <= 64) stats->history[iters - 1] = rel;
          continue;
        }
        done = true;
        return CDL_OK;
      }
      if (iters >= opts->max_iter || !(rel <= 1e6)) done = true;   // NaN or growing: no contraction
      return CDL_OK;
    }
  }

  // x = D^{-1/2} R in the chain's working precision (and its bf16 operand)
  int precond_in() {
    {
      const size_t cnt = (size_t)np * kp;
      Launch L(ctx, CDL_KC_MISC, 0);
      if (ch->dtype == CDL_F64)
        k_precond_in<double><<<blocks_for(cnt, 256), 256, 0, st>>>(R, ch->rsqrt_d, n, k, np, kp,
                                                                    static_cast<double*>(vx));
      else
        k_precond_in<float><<<blocks_for(cnt, 256), 256, 0, st>>>(R, ch->rsqrt_d, n, k, np, kp,
                                                                   static_cast<float*>(vx));
      CDL_TRY(L.done());
    }
    if (bf16) {
      dim3 g((np + 31) / 32, (kp + 31) / 32);
      Launch L(ctx, CDL_KC_MISC, 0);
      k_update_bf16<<<g, 256, 0, st>>>(static_cast<float*>(vx), nullptr, 0, np, kp,
                                       static_cast<__nv_bfloat16*>(vxop), 0);
      CDL_TRY(L.done());
    }
    return CDL_OK;
  }

  // x <- (I + S~_lvl) x
  int apply_level(int lvl) {
    if (bf16) {
      CDL_TRY(apply_tc(ctx, ch, lvl, vxop, static_cast<float*>(vpart), kp, splits));
      dim3 g((np + 31) / 32, (kp + 31) / 32);
      Launch L(ctx, CDL_KC_MISC, 0);
      k_update_bf16<<<g, 256, 0, st>>>(static_cast<float*>(vx), static_cast<const float*>(vpart), splits, np, kp,
                                       static_cast<__nv_bfloat16*>(vxop), 1);
      return L.done();
    }
    CDL_TRY(apply_simt(ctx, ch, lvl, vx, vpart, kp, splits));
    const size_t cnt = (size_t)np * kp;
    Launch L(ctx, CDL_KC_MISC, 0);
    if (ch->dtype == CDL_F64)
      k_update_simt<double><<<blocks_for(cnt, 256), 256, 0, st>>>(
          static_cast<double*>(vx), static_cast<const double*>(vpart), splits, cnt);
    else
      k_update_simt<float><<<blocks_for(cnt, 256), 256, 0, st>>>(
          static_cast<float*>(vx), static_cast<const float*>(vpart), splits, cnt);
    return L.done();
  }

  // Z += D^{-1/2} x, D-weighted centring, then the residual (in full on the
  // first step or always_full, else recursively) and its norm.
  int finish_step(bool always_full) {
    {
      Launch L(ctx, CDL_KC_MISC, 0);
      if (ch->dtype == CDL_F64)
        k_precond_out<double><<<blocks_for((size_t)np * kp, 256), 256, 0, st>>>(
            static_cast<const double*>(vx), ch->rsqrt_d, n, k, np, kp, Z, static_cast<float*>(vdz));
      else
        k_precond_out<float><<<blocks_for((size_t)np * kp, 256), 256, 0, st>>>(
            static_cast<const float*>(vx), ch->rsqrt_d, n, k, np, kp, Z, static_cast<float*>(vdz));
      CDL_TRY(L.done());
    }
    {
      dim3 g(cs_parts, (k + 255) / 256);
      Launch L(ctx, CDL_KC_MISC, 0);
      k_colsum_dz<<<g, 256, 0, st>>>(Z, ch->D, n, k, cs_rows, static_cast<double*>(vcs));
      CDL_TRY(L.done());
    }
    {
      double* shift = static_cast<double*>(vcs) + (size_t)cs_parts * k;
      {
        Launch L(ctx, CDL_KC_MISC, 0);
        k_center_shift<<<(k + 255) / 256, 256, 0, st>>>(static_cast<const double*>(vcs), cs_parts, k, ch->vol, shift);
        CDL_TRY(L.done());
      }
      Launch L(ctx, CDL_KC_MISC, 0);
      k_center<<<blocks_for(nk, 256), 256, 0, st>>>(Z, shift, n, k);
      CDL_TRY(L.done());
    }
    ++iters;
    const double prev = rel;
    if (iters == 1 || always_full) {
      CDL_TRY(full_residual());
      exact_r = true;
      drift = 0.0;
    } else {
      CDL_TRY(update_residual());
      drift += 1e-5 * rel;   // error of the L dZ product (16-bit operands or float32), |L dZ| ~ |R| before
      exact_r = false;
    }
    CDL_TRY(read_norm());
    if (!exact_r && rel > 0.5 * prev) {
      // a recursive residual that stops falling is dominated by its own
      // rounding: form it again in full
      CDL_TRY(full_residual());
      CDL_TRY(read_norm());
      exact_r = true;
      drift = 0.0;
    }
    if (stats && iters <= 64) stats->history[iters - 1] = rel;
    return CDL_OK;
  }

  int status(const cdl_solve_opts* opts) const {
    if (!(rel <= 1e6)) return CDL_ERR_NOT_CONVERGED;
    return (opts->rel_tol > 0 && !(rel <= opts->rel_tol)) ? CDL_ERR_NOT_CONVERGED : CDL_OK;
  }
};

// columns c0 .. c0 + kb - 1 of the n x k matrix Y into the n x kb matrix Yb, and back
__global__ void k_gather_cols(const double* __restrict__ Y, int n, int k, int c0, int kb, double* __restrict__ Yb) {
  const size_t cnt = (size_t)n * kb;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / kb;
    Yb[e] = Y[i * k + c0 + (e - i * kb)];
  }
}

__global__ void k_scatter_cols(const double* __restrict__ Zb, int n, int kb, int c0, int k, double* __restrict__ Z) {
  const size_t cnt = (size_t)n * kb;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / kb;
    Z[i * k + c0 + (e - i * kb)] = Zb[e];
  }
}

}  // namespace

// The tensor-core apply multiplies a level by at most 128 right-hand sides
// (MMA N = 2 kp <= 256 for the hi and lo halves). Alg. 2's Richardson
// iteration and the chain apply act on each column on its own, so more
// columns are solved as blocks of at most 128, each with its own float64
// residual and its own stopping test against its own ||Y_b||; the blocks
// step together, and each level is applied to every block still running
// while it is loaded (levels in host memory cross the link once per step,
// not once per block). The reported residual is the one of all k columns,
// sqrt(sum_b ||R_b||^2 / sum_b ||Y_b||^2), below rel_tol when every block
// is; iters is the largest block count and history[t] combines the blocks'
// residuals after t + 1 steps (a block that stopped earlier keeps its last).
int chain_solve(cdl_ctx* ctx, const cdl_chain* ch, const double* A, const double* Y, int k,
                const cdl_solve_opts* opts, double* Z, cdl_solve_stats* stats) {
  const bool tensor = ch->dtype == CDL_BF16 || ch->dtype == CDL_FP8E4M3 || ch->dtype == CDL_FP8E4M3_T128;
  const int nblk = (tensor && k > 128) ? (k + 127) / 128 : 1;
  const int kb_max = nblk == 1 ? k : (int)round_up((k + nblk - 1) / nblk, 16);
  const int n = (int)ch->n;
  cudaStream_t st = ctx->stream;
  std::vector<SolveBlock> B(nblk);
  std::vector<cdl_solve_stats> bst(nblk);
  const unsigned gb = (unsigned)std::min<size_t>(((size_t)n * kb_max + 255) / 256, (size_t)ctx->sm_count * 8);
  for (int b = 0; b < nblk; ++b) {
    SolveBlock& s = B[b];
    s.ctx = ctx;
    s.ch = ch;
    s.A = A;
    const int c0 = b * kb_max;
    s.k = std::min(kb_max, k - c0);
    if (nblk == 1) {
      s.Y = Y;
      s.Z = Z;
      s.stats = stats;
    } else {
      void *vyb, *vzb;
      CDL_TRY(ws_get(ctx, ("solve.block_y#" + std::to_string(b)).c_str(), (size_t)n * kb_max * 8, &vyb));
      CDL_TRY(ws_get(ctx, ("solve.block_z#" + std::to_string(b)).c_str(), (size_t)n * kb_max * 8, &vzb));
      s.Y = static_cast<double*>(vyb);
      s.Z = static_cast<double*>(vzb);
      s.stats = &bst[b];
      Launch L(ctx, CDL_KC_MISC, 0);
      k_gather_cols<<<gb, 256, 0, st>>>(Y, n, k, c0, s.k, static_cast<double*>(vyb));
      CDL_TRY(L.done());
    }
    CDL_TRY(s.init(b));
  }
  // a regenerated graph keeps no A operand for the recursive update
  const bool always_full = (opts->flags & CDL_SOLVE_FULL_RESIDUAL) != 0 || ch->regen != nullptr;
  while (true) {
    std::vector<SolveBlock*> run;
    for (SolveBlock& s : B) {
      if (s.done) continue;
      CDL_TRY(s.pre_step(opts));
      if (!s.done) run.push_back(&s);
    }
    if (run.empty()) break;
    for (SolveBlock* s : run) CDL_TRY(s->precond_in());
    for (int lvl = 0; lvl < ch->d_eff; ++lvl)
      for (SolveBlock* s : run) CDL_TRY(s->apply_level(lvl));
    for (SolveBlock* s : run) CDL_TRY(s->finish_step(always_full));
  }
  if (nblk == 1) {
    if (stats) {
      stats->iters = B[0].iters;
      stats->rel_res = B[0].rel;
    }
    return B[0].status(opts);
  }
  double yy_all = 0.0, rr_all = 0.0;
  double hist_rr[64] = {0};
  int iters = 0, status = CDL_OK;
  for (int b = 0; b < nblk; ++b) {
    const SolveBlock& s = B[b];
    if (s.status(opts) != CDL_OK) status = CDL_ERR_NOT_CONVERGED;
    {
      Launch L(ctx, CDL_KC_MISC, 0);
      k_scatter_cols<<<gb, 256, 0, st>>>(s.Z, n, s.k, b * kb_max, k, Z);
      CDL_TRY(L.done());
    }
    yy_all += s.yy;
    rr_all += s.rel * s.rel * s.yy;
    iters = std::max(iters, s.iters);
    for (int t = 0; t < 64; ++t) {
      const double h = t < s.iters ? bst[b].history[t] : s.rel;
      hist_rr[t] += h * h * s.yy;
    }
  }
  if (stats) {
    stats->iters = iters;
    stats->rel_res = yy_all > 0 ? std::sqrt(rr_all / yy_all) : 0.0;
    for (int t = 0; t < 64; ++t)
      stats->history[t] = (t < iters && yy_all > 0) ? std::sqrt(hist_rr[t] / yy_all) : 0.0;
  }
  CDL_CUDA_TRY(cudaStreamSynchronize(st));
  return status;
}

void batch_residual_tile(int k, int* tm, int* tn) {
  *tm = 128;
  *tn = (k + 31) / 32 * 32;
}

namespace {
template <typename K, typename... Args>
int run_tiles(cdl_ctx* ctx, const BatchSolve& B, K kern, const BTiles& t, int kc, double work, Args... args) {
  if (t.count == 0) return CDL_OK;
  Launch L(ctx, kc, work);
  kern<<<t.count, 256, 0, ctx->stream>>>(t.p, B.gs, args...);
  return L.done();
}
}  // namespace

int batch_solve_start(cdl_ctx* ctx, const BatchSolve& B) {
  CDL_TRY(run_tiles(ctx, B, k_b_start, B.elem, CDL_KC_MISC, 0.0, B.k));
  Launch L(ctx, CDL_KC_MISC, 0);
  k_b_begin<<<B.G2, 256, 0, ctx->stream>>>(B.gs, B.st);
  return L.done();
}

int batch_solve_slot(cdl_ctx* ctx, const BatchSolve& B) {
  const BState* cst = B.st;
  CDL_CUDA_TRY(cudaMemsetAsync(B.active, 0, sizeof(int), ctx->stream));
  CDL_TRY(run_tiles(ctx, B, k_b_precond_in, B.t32, CDL_KC_MISC, 0.0, cst, B.k, B.kp));
  for (int lvl = 0; lvl < B.d; ++lvl) {
    CDL_TRY(tc_apply_grouped(ctx, B.lvl_first + lvl, B.lvl_groups + (size_t)lvl * B.G2, B.apply.p, B.apply.count,
                             B.kp, CMD_STEP, CDL_KC_APPLY, B.apply_bytes));
    CDL_TRY(run_tiles(ctx, B, k_b_update, B.t32, CDL_KC_MISC, 0.0, cst, B.kp));
  }
  CDL_TRY(run_tiles(ctx, B, k_b_precond_out, B.t32, CDL_KC_MISC, 0.0, cst, B.k, B.kp));
  CDL_TRY(run_tiles(ctx, B, k_b_colsum, B.cs, CDL_KC_MISC, 0.0, cst, B.k));
  CDL_TRY(run_tiles(ctx, B, k_b_center, B.elem, CDL_KC_MISC, 0.0, cst, B.k));
  // full residual (first step, certification) on the tensor cores from exact
  // slices, or the recursive update
  CDL_CUDA_TRY(cudaMemsetAsync(B.zmax_all, 0, B.zmax_bytes, ctx->stream));
  CDL_TRY(run_tiles(ctx, B, k_b_zcolmax, B.elem, CDL_KC_MISC, 0.0, cst, B.k));
  CDL_TRY(run_tiles(ctx, B, k_b_zslice, B.zst, CDL_KC_MISC, 0.0, cst, B.k));
  CDL_TRY(resid_tc_grouped(ctx, B.rgroups, B.runits.p, B.runits.count, B.kg, CMD_FULL, B.resid_work));
  CDL_TRY(run_tiles(ctx, B, k_b_resid_combine, B.elem, CDL_KC_RESIDUAL, 0.0, cst, B.k));
  if (!B.always_full) {
    CDL_TRY(tc_apply_grouped(ctx, B.res_first, B.res_groups, B.apply.p, B.apply.count, B.kp, CMD_RECUR,
                             CDL_KC_RESIDUAL, 0.0));
    CDL_TRY(tc_apply_grouped(ctx, B.res_first + 1, B.res_groups + B.G2, B.apply.p, B.apply.count, B.kp, CMD_RECUR,
                             CDL_KC_RESIDUAL, 0.0));
    CDL_TRY(run_tiles(ctx, B, k_b_residual_update, B.elem, CDL_KC_RESIDUAL, 0.0, cst, B.k, B.kp));
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_b_decide<<<B.G2, 256, 0, ctx->stream>>>(B.gs, B.st, B.rel_tol, B.max_iter, B.always_full ? 1 : 0, B.active);
  return L.done();
}

}  // namespace cdl
