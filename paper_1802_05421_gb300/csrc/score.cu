// CAD node scores and top anomalies (Alg. 4; edge score of Sec. 2):
//   F_i = sum_{j != i} |A1_ij - A2_ij| |c2(i,j) - c1(i,j)|,
//   c_t(i,j) = vol_t ||Z_t[i,:] - Z_t[j,:]||^2.
// The commute-time difference is formed without cancelling the two commute
// times: with a = sqrt(vol2) Z2 - sqrt(vol1) Z1 and b = sqrt(vol2) Z2 +
// sqrt(vol1) Z1, c2 - c1 = (a_i - a_j).(b_i - b_j). The k-term sum itself
// still cancels (its terms have both signs), so the float32 variant keeps
// every term to about 2^-45 of its column's scale: a and b are split on a
// per-column fixed grid into hi + lo, with hi on a grid fine enough for 23
// bits of the column maximum, so that hi_i - hi_j is exact in float32;
// products are made exact with a fused multiply-add and the sum is
// compensated (TwoSum, Knuth), as in the doubled-precision dot product of
// Ogita, Rump and Oishi (2005).
// Each unordered pair (i < j) is visited once in 64 x 64 upper-triangle
// tiles; the two row contributions of a tile go to a per-(partner block, node)
// slot, and F is the fixed-order sum of those slots (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "tiles.cuh"

namespace cdl {
namespace {

constexpr int ST = 64;   // pair tile
constexpr int RC = 8;    // projection rows per smem chunk

// Column maxima of |a| and |b| (cmax[r], cmax[k + r]; float bits, rounded up
// by 2^-20 so that they bound the float64 values).
__device__ __forceinline__ void score_colmax(const double* __restrict__ Z1, const double* __restrict__ Z2,
                                             const double* __restrict__ vol1, const double* __restrict__ vol2,
                                             int n, int k, unsigned* __restrict__ cmax, size_t idx) {
  if (idx >= (size_t)n * k) return;
  const int r = (int)(idx % k);
  const double s1 = sqrt(*vol1), s2 = sqrt(*vol2);
  const double w = s2 * Z2[idx], v = s1 * Z1[idx];
  const float fa = (float)(fabs(w - v) * (1.0 + 0x1p-20)), fb = (float)(fabs(w + v) * (1.0 + 0x1p-20));
  atomicMax(cmax + r, __float_as_uint(fa));        // non-negative floats order as their bits
  atomicMax(cmax + k + r, __float_as_uint(fb));
}

// x = hi + lo with hi on the grid q = 2^(e - 21), 2^e <= M < 2^(e+1) the
// column bound: |hi| / q <= 2^22 + 1, so differences of two hi values are
// exact in float32; lo = x - hi (|lo| <= q / 2) rounded to float32.
__device__ __forceinline__ void grid_split(double x, unsigned mbits, float& hi, float& lo) {
  const int e = (int)((mbits >> 23) & 0xFF) - 127;
  if (e < -90) {   // column of (near) zeros
    hi = (float)x;
    lo = 0.f;
    return;
  }
  const double q = ldexp(1.0, e - 21);
  const double h = rint(x / q) * q;
  hi = (float)h;
  lo = (float)(x - h);
}

// aT/bT hi/lo, stored transposed (k x n) for coalesced tile loads.
__device__ __forceinline__ void score_prep(const double* __restrict__ Z1, const double* __restrict__ Z2,
                                           const double* __restrict__ vol1, const double* __restrict__ vol2, int n,
                                           int k, const unsigned* __restrict__ cmax, float* __restrict__ ah,
                                           float* __restrict__ al, float* __restrict__ bh, float* __restrict__ bl,
                                           size_t idx) {
  if (idx >= (size_t)n * k) return;
  const int i = (int)(idx / k), r = (int)(idx % k);
  const double s1 = sqrt(*vol1), s2 = sqrt(*vol2);
  const double w = s2 * Z2[idx], v = s1 * Z1[idx];
  const size_t o = (size_t)r * n + i;
  grid_split(w - v, cmax[r], ah[o], al[o]);
  grid_split(w + v, cmax[k + r], bh[o], bl[o]);
}

__global__ void k_score_colmax(const double* __restrict__ Z1, const double* __restrict__ Z2,
                               const double* __restrict__ vol1, const double* __restrict__ vol2, int n, int k,
                               unsigned* __restrict__ cmax) {
  score_colmax(Z1, Z2, vol1, vol2, n, k, cmax, blockIdx.x * (size_t)blockDim.x + threadIdx.x);
}

__global__ void k_score_prep(const double* __restrict__ Z1, const double* __restrict__ Z2,
                             const double* __restrict__ vol1, const double* __restrict__ vol2, int n, int k,
                             const unsigned* __restrict__ cmax, float* __restrict__ ah, float* __restrict__ al,
                             float* __restrict__ bh, float* __restrict__ bl) {
  score_prep(Z1, Z2, vol1, vol2, n, k, cmax, ah, al, bh, bl, blockIdx.x * (size_t)blockDim.x + threadIdx.x);
}

// float64 variant: aT, bT (k x n).
__device__ __forceinline__ void score_prep64(const double* __restrict__ Z1, const double* __restrict__ Z2,
                                             const double* __restrict__ vol1, const double* __restrict__ vol2,
                                             int n, int k, double* __restrict__ aT, double* __restrict__ bT,
                                             size_t idx) {
  if (idx >= (size_t)n * k) return;
  const int i = (int)(idx / k), r = (int)(idx % k);
  const double s1 = sqrt(*vol1), s2 = sqrt(*vol2);
  const double w = s2 * Z2[idx], v = s1 * Z1[idx];
  const size_t o = (size_t)r * n + i;
  aT[o] = w - v;
  bT[o] = w + v;
}

__global__ void k_score_prep64(const double* __restrict__ Z1, const double* __restrict__ Z2,
                               const double* __restrict__ vol1, const double* __restrict__ vol2, int n, int k,
                               double* __restrict__ aT, double* __restrict__ bT) {
  score_prep64(Z1, Z2, vol1, vol2, n, k, aT, bT, blockIdx.x * (size_t)blockDim.x + threadIdx.x);
}


// Per-tile accumulation of |A1 - A2| |c2 - c1| into row and column partials.
__device__ __forceinline__ void tile_finish(const double* __restrict__ A1, const double* __restrict__ A2,
                                            int n, int i0, int j0, int bi, int bj, int tx, int ty,
                                            const double (&dc)[4][4], double* __restrict__ contrib,
                                            double (*rsum)[17], double (*csum)[17], double* __restrict__ Eout) {
  double rpart[4] = {0, 0, 0, 0}, cpart[4] = {0, 0, 0, 0};
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty * 4 + u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx * 4 + v;
      if (i < n && j < n && (bi != bj || i < j)) {
        const size_t o = (size_t)i * n + j;
        const double e = fabs(A1[o] - A2[o]) * fabs(dc[u][v]);
        if (Eout) Eout[o] = e;   // edge score of (i, j), i < j
        rpart[u] += e;
        cpart[v] += e;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) rsum[ty * 4 + u][tx] = rpart[u];
#pragma unroll
  for (int v = 0; v < 4; ++v) csum[tx * 4 + v][ty] = cpart[v];
  __syncthreads();
  const int tid = threadIdx.x;
  if (tid < ST) {
    double rs = 0.0, cs = 0.0;
    for (int q = 0; q < 16; ++q) {
      rs += rsum[tid][q];
      cs += csum[tid][q];
    }
    const int i = i0 + tid, j = j0 + tid;
    if (bi == bj) {
      if (i < n) contrib[(size_t)bi * n + i] = rs + cs;
    } else {
      if (i < n) contrib[(size_t)bj * n + i] = rs;   // row i, partner block bj
      if (j < n) contrib[(size_t)bi * n + j] = cs;   // node j, partner block bi
    }
  }
}

__device__ __forceinline__ void score_tile(const double* __restrict__ A1, const double* __restrict__ A2,
                                           const float* __restrict__ ah, const float* __restrict__ al,
                                           const float* __restrict__ bh, const float* __restrict__ bl, int n, int k,
                                           double* __restrict__ contrib, int bi, int bj,
                                           double* __restrict__ Eout = nullptr) {
  __shared__ __align__(16) float sI[4][RC][ST];   // ah, al, bh, bl of the row block
  __shared__ __align__(16) float sJ[4][RC][ST];   // ... of the column block
  __shared__ double rsum[ST][17];
  __shared__ double csum[ST][17];
  const int i0 = bi * ST, j0 = bj * ST;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4], cmp[4][4];   // compensated sum: acc + cmp
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = cmp[u][v] = 0.f;
  const float* src[4] = {ah, al, bh, bl};
  for (int r0 = 0; r0 < k; r0 += RC) {
    for (int e = tid; e < RC * ST; e += 256) {
      const int rr = e / ST, c = e % ST;
      const int r = r0 + rr;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sI[q][rr][c] = (r < k && i0 + c < n) ? src[q][(size_t)r * n + i0 + c] : 0.f;
        sJ[q][rr][c] = (r < k && j0 + c < n) ? src[q][(size_t)r * n + j0 + c] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < RC; ++rr) {
      const float4 iah = *reinterpret_cast<const float4*>(&sI[0][rr][ty * 4]);
      const float4 ial = *reinterpret_cast<const float4*>(&sI[1][rr][ty * 4]);
      const float4 ibh = *reinterpret_cast<const float4*>(&sI[2][rr][ty * 4]);
      const float4 ibl = *reinterpret_cast<const float4*>(&sI[3][rr][ty * 4]);
      const float4 jah = *reinterpret_cast<const float4*>(&sJ[0][rr][tx * 4]);
      const float4 jal = *reinterpret_cast<const float4*>(&sJ[1][rr][tx * 4]);
      const float4 jbh = *reinterpret_cast<const float4*>(&sJ[2][rr][tx * 4]);
      const float4 jbl = *reinterpret_cast<const float4*>(&sJ[3][rr][tx * 4]);
      const float Iah[4] = {iah.x, iah.y, iah.z, iah.w}, Ial[4] = {ial.x, ial.y, ial.z, ial.w};
      const float Ibh[4] = {ibh.x, ibh.y, ibh.z, ibh.w}, Ibl[4] = {ibl.x, ibl.y, ibl.z, ibl.w};
      const float Jah[4] = {jah.x, jah.y, jah.z, jah.w}, Jal[4] = {jal.x, jal.y, jal.z, jal.w};
      const float Jbh[4] = {jbh.x, jbh.y, jbh.z, jbh.w}, Jbl[4] = {jbl.x, jbl.y, jbl.z, jbl.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float dah = __fsub_rn(Iah[u], Jah[v]);   // exact (grid split)
          const float dal = __fsub_rn(Ial[u], Jal[v]);
          const float dbh = __fsub_rn(Ibh[u], Jbh[v]);   // exact
          const float dbl = __fsub_rn(Ibl[u], Jbl[v]);
          const float p = __fmul_rn(dah, dbh);
          float x = __fmaf_rn(dah, dbh, -p);             // p + x = dah dbh exactly
          x = __fmaf_rn(dah, dbl, x);
          x = __fmaf_rn(dal, dbh, x);
          const float t = __fadd_rn(acc[u][v], p);       // TwoSum(acc, p)
          const float z = __fsub_rn(t, acc[u][v]);
          const float err = __fadd_rn(__fsub_rn(acc[u][v], __fsub_rn(t, z)), __fsub_rn(p, z));
          acc[u][v] = t;
          cmp[u][v] = __fadd_rn(cmp[u][v], __fadd_rn(err, x));
        }
    }
    __syncthreads();
  }
  double dc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) dc[u][v] = (double)acc[u][v] + (double)cmp[u][v];
  tile_finish(A1, A2, n, i0, j0, bi, bj, tx, ty, dc, contrib, rsum, csum, Eout);
}

__global__ void __launch_bounds__(256) k_score_pairs(const double* __restrict__ A1, const double* __restrict__ A2,
                                                      const float* __restrict__ ah, const float* __restrict__ al,
                                                      const float* __restrict__ bh, const float* __restrict__ bl,
                                                      int n, int k, double* __restrict__ contrib) {
  const int nb = (n + ST - 1) / ST;
  int bi, bj;
  block_tri_index(nb, bi, bj);
  score_tile(A1, A2, ah, al, bh, bl, n, k, contrib, bi, bj);
}

// float64 variant: c2 - c1 = sum_r (a_ir - a_jr)(b_ir - b_jr) in float64.
__device__ __forceinline__ void score_tile64(const double* __restrict__ A1, const double* __restrict__ A2,
                                             const double* __restrict__ aT, const double* __restrict__ bT, int n,
                                             int k, double* __restrict__ contrib, int bi, int bj,
                                             double* __restrict__ Eout = nullptr) {
  __shared__ __align__(16) double sI[2][RC][ST];
  __shared__ __align__(16) double sJ[2][RC][ST];
  __shared__ double rsum[ST][17];
  __shared__ double csum[ST][17];
  const int i0 = bi * ST, j0 = bj * ST;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  const double* src[2] = {aT, bT};
  for (int r0 = 0; r0 < k; r0 += RC) {
    for (int e = tid; e < RC * ST; e += 256) {
      const int rr = e / ST, c = e % ST;
      const int r = r0 + rr;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        sI[q][rr][c] = (r < k && i0 + c < n) ? src[q][(size_t)r * n + i0 + c] : 0.0;
        sJ[q][rr][c] = (r < k && j0 + c < n) ? src[q][(size_t)r * n + j0 + c] : 0.0;
      }
    }
    __syncthreads();
    for (int rr = 0; rr < RC; ++rr) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const double da = sI[0][rr][ty * 4 + u] - sJ[0][rr][tx * 4 + v];
          const double db = sI[1][rr][ty * 4 + u] - sJ[1][rr][tx * 4 + v];
          acc[u][v] = fma(da, db, acc[u][v]);
        }
    }
    __syncthreads();
  }
  tile_finish(A1, A2, n, i0, j0, bi, bj, tx, ty, acc, contrib, rsum, csum, Eout);
}

__global__ void __launch_bounds__(256) k_score_pairs64(const double* __restrict__ A1,
                                                        const double* __restrict__ A2,
                                                        const double* __restrict__ aT,
                                                        const double* __restrict__ bT, int n, int k,
                                                        double* __restrict__ contrib) {
  const int nb = (n + ST - 1) / ST;
  int bi, bj;
  block_tri_index(nb, bi, bj);
  score_tile64(A1, A2, aT, bT, n, k, contrib, bi, bj);
}


__global__ void k_score_reduce(const double* __restrict__ contrib, int nb, int n, double* __restrict__ F) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += contrib[(size_t)b * n + i];
  F[i] = s;
}

// ---- tensor-core scores (score dtype bf16): slices of u = [a / g | b g] and
// v = [b g | a / g], and d_i = a_i.b_i, for score_tc.
__device__ __forceinline__ void tcs_ab(const double* __restrict__ Z1, const double* __restrict__ Z2, double s1,
                                       double s2, size_t idx, double& a, double& b) {
  const double w = s2 * Z2[idx], v = s1 * Z1[idx];
  a = w - v;
  b = w + v;
}

// column maxima of |a| (cm[r]) and |b| (cm[k + r]) as float64 bits: maxima of
// a row chunk per block in shared memory, then one global atomic per column
// and block (k <= 1024)
__global__ void __launch_bounds__(256) k_tcs_colmax(const double* __restrict__ Z1, const double* __restrict__ Z2,
                                                     const double* __restrict__ vol1, const double* __restrict__ vol2,
                                                     int n, int k, unsigned long long* __restrict__ cm) {
  __shared__ unsigned long long sm[2048];
  for (int c = threadIdx.x; c < 2 * k; c += blockDim.x) sm[c] = 0ull;
  __syncthreads();
  const double s1 = sqrt(*vol1), s2 = sqrt(*vol2);
  const int rows_per_block = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
  for (size_t idx = (size_t)r0 * k + threadIdx.x; idx < (size_t)r1 * k; idx += blockDim.x) {
    double a, b;
    tcs_ab(Z1, Z2, s1, s2, idx, a, b);
    const int r = (int)(idx % k);
    atomicMax(sm + r, (unsigned long long)__double_as_longlong(fabs(a)));
    atomicMax(sm + k + r, (unsigned long long)__double_as_longlong(fabs(b)));
  }
  __syncthreads();
  for (int c = threadIdx.x; c < 2 * k; c += blockDim.x)
    if (sm[c]) atomicMax(cm + c, sm[c]);
}

// g_r = 2^e_r with e_r = floor((E(max|a_r|) - E(max|b_r|)) / 2) (E: binary
// exponent), so that a / g and b g have maxima within a factor of 4; c = twice
// the power of two strictly above every |a / g|, |b g| (cs[0]: every value
// divided by c is below 1/2) and cs[1] = c^2 2^-48, the unit of M and d. One
// block.
__global__ void k_tcs_scales(const unsigned long long* __restrict__ cm, int k, double* __restrict__ g,
                             double* __restrict__ cs) {
  __shared__ int emax[256];
  int em = -1100;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const unsigned long long ba = cm[r], bb = cm[k + r];
    int e = 0;
    if (ba != 0 && bb != 0) {
      const int ea = (int)((ba >> 52) & 0x7FF) - 1023, eb = (int)((bb >> 52) & 0x7FF) - 1023;
      e = (ea - eb) >> 1;                                   // floor
    }
    g[r] = ldexp(1.0, e);
    const double ma = __longlong_as_double((long long)ba) * ldexp(1.0, -e);
    const double mb = __longlong_as_double((long long)bb) * ldexp(1.0, e);
    const double mx = fmax(ma, mb);
    if (mx > 0.0) em = max(em, (int)((__double_as_longlong(mx) >> 52) & 0x7FF) - 1023);
  }
  emax[threadIdx.x] = em;
  __syncthreads();
  if (threadIdx.x == 0) {
    int e = -1100;
    for (int t = 0; t < (int)blockDim.x; ++t) e = max(e, emax[t]);
    if (e < -1000) e = 0;                                   // all zero
    cs[0] = ldexp(1.0, e + 2);                              // 2^E <= max < 2^(E+1) = c / 2
    cs[1] = ldexp(1.0, 2 * (e + 2) - 48);
  }
}

// Six planes (rows x k2p bf16) each of u / c and v / c: signed base-256
// digits of the values rounded to 2^-48 (|value| < 1/2: every digit at most
// 128 in magnitude), plane t holding digit t times 2^-8t; zero padded.
__global__ void __launch_bounds__(256) k_tcs_slice(const double* __restrict__ Z1, const double* __restrict__ Z2,
                                                    const double* __restrict__ vol1, const double* __restrict__ vol2,
                                                    int n, int k, int rows, int k2p, const double* __restrict__ g,
                                                    const double* __restrict__ cs, __nv_bfloat16* __restrict__ U,
                                                    __nv_bfloat16* __restrict__ V) {
  const double s1 = sqrt(*vol1), s2 = sqrt(*vol2);
  const double rc = 1.0 / cs[0];                            // power of two: exact
  const size_t plane = (size_t)rows * k2p;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k2p), col = (int)(idx % k2p);
    long long Nu = 0, Nv = 0;
    if (i < n && col < 2 * k) {
      const int r = col < k ? col : col - k;
      double a, b;
      tcs_ab(Z1, Z2, s1, s2, (size_t)i * k + r, a, b);
      const double at = a / g[r], bt = b * g[r];            // powers of two: exact
      const double xu = col < k ? at : bt, xv = col < k ? bt : at;
      Nu = llrint(xu * rc * 0x1p48);
      Nv = llrint(xv * rc * 0x1p48);
    }
#pragma unroll
    for (int t = 1; t <= 6; ++t) {
      const int sh = 48 - 8 * t;
      long long du = Nu, dv = Nv;
      if (sh > 0) {
        du = (Nu + (1LL << (sh - 1))) >> sh;
        dv = (Nv + (1LL << (sh - 1))) >> sh;
      }
      Nu -= du << sh;
      Nv -= dv << sh;
      U[(size_t)(t - 1) * plane + idx] = __float2bfloat16_rn(ldexpf((float)du, -8 * t));
      V[(size_t)(t - 1) * plane + idx] = __float2bfloat16_rn(ldexpf((float)dv, -8 * t));
    }
  }
}

// d_i = sum_r a_ir b_ir (float64, columns in order), in units of c^2 2^-48,
// one warp per row (padded rows 0).
__global__ void __launch_bounds__(256) k_tcs_diag(const double* __restrict__ Z1, const double* __restrict__ Z2,
                                                   const double* __restrict__ vol1, const double* __restrict__ vol2,
                                                   int n, int k, int rows, const double* __restrict__ cs,
                                                   long long* __restrict__ dint) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= rows) return;
  const double s1 = sqrt(*vol1), s2 = sqrt(*vol2);
  double acc = 0.0;
  if (row < n)
    for (int r = lane; r < k; r += 32) {
      double a, b;
      tcs_ab(Z1, Z2, s1, s2, (size_t)row * k + r, a, b);
      acc = fma(a, b, acc);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) dint[row] = llrint(acc / cs[1]);           // division by a power of two: exact
}

// (v, i) precedes (w, j) in the anomaly order: larger score first, then the
// lower index.
__device__ __forceinline__ bool better(double v, int i, double w, int j) {
  return v > w || (v == w && i < j);
}

__device__ __forceinline__ void topk_block(const double* __restrict__ F, int n, int topk,
                                           int64_t* __restrict__ out) {
  __shared__ double sv[32];
  __shared__ int si[32];
  double pv = INFINITY;
  int pi = -1;
  for (int t = 0; t < topk; ++t) {
    double bv = -INFINITY;
    int bidx = INT_MAX;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = F[i];
      const bool after = v < pv || (v == pv && i > pi);
      if (after && better(v, i, bv, bidx)) {
        bv = v;
        bidx = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (better(ov, oi, bv, bidx)) {
        bv = ov;
        bidx = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      sv[threadIdx.x >> 5] = bv;
      si[threadIdx.x >> 5] = bidx;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      bv = threadIdx.x < (blockDim.x >> 5) ? sv[threadIdx.x] : -INFINITY;
      bidx = threadIdx.x < (blockDim.x >> 5) ? si[threadIdx.x] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (better(ov, oi, bv, bidx)) {
          bv = ov;
          bidx = oi;
        }
      }
      if (threadIdx.x == 0) {
        sv[0] = bv;
        si[0] = bidx;
        out[t] = bidx == INT_MAX ? -1 : bidx;
      }
    }
    __syncthreads();
    pv = sv[0];
    pi = si[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_topk(const double* __restrict__ F, int n, int topk,
                                                int64_t* __restrict__ out) {
  topk_block(F, n, topk, out);
}

// ---------------------------------------------------------------- anomalous edge set
// CAD's anomalous edges (Sec. 3.3): the smallest set of edges whose removal
// leaves a remaining total change Delta E below delta. Taking edges in
// descending Delta E (ties by (i, j)) is optimal for that cardinality
// problem, so the set is {Delta E > tau} plus the first c edges equal to
// tau, for the largest tau whose set {Delta E >= tau} already suffices. tau
// is found by bisection on the float64 bit patterns (non-negative doubles
// order like their bits), each step a fixed-order sum over the upper
// triangle, so the result does not depend on scheduling.

__global__ void __launch_bounds__(256) k_edge_pairs(const double* __restrict__ A1, const double* __restrict__ A2,
                                                     const void* __restrict__ ab, int n, int k, int fp64,
                                                     double* __restrict__ contrib, double* __restrict__ E) {
  const int nb = (n + ST - 1) / ST;
  int bi, bj;
  block_tri_index(nb, bi, bj);
  const size_t nk = (size_t)n * k;
  if (fp64) {
    const double* aT = static_cast<const double*>(ab);
    score_tile64(A1, A2, aT, aT + nk, n, k, contrib, bi, bj, E);
  } else {
    const float* ah = static_cast<const float*>(ab);
    score_tile(A1, A2, ah, ah + nk, ah + 2 * nk, ah + 3 * nk, n, k, contrib, bi, bj, E);
  }
}

__device__ __forceinline__ unsigned long long dkey(double v) { return (unsigned long long)__double_as_longlong(v); }

// Per-block sums and counts of the upper-triangle entries with key >= tau
// (rows i = block, block + grid, ...; fixed order).
__global__ void __launch_bounds__(256) k_edge_mass(const double* __restrict__ E, int n, unsigned long long tau,
                                                    double* __restrict__ psum, unsigned long long* __restrict__ pcnt) {
  __shared__ double rs[8];
  __shared__ unsigned long long rc[8];
  double s = 0.0;
  unsigned long long c = 0;
  for (int i = blockIdx.x; i < n - 1; i += gridDim.x)
    for (int j = i + 1 + threadIdx.x; j < n; j += 256) {
      const double v = E[(size_t)i * n + j];
      if (dkey(v) >= tau) {
        s += v;
        ++c;
      }
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rs[threadIdx.x >> 5] = s;
    rc[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    unsigned long long u = 0;
    for (int w = 0; w < 8; ++w) {
      t += rs[w];
      u += rc[w];
    }
    psum[blockIdx.x] = t;
    pcnt[blockIdx.x] = u;
  }
}

__global__ void k_edge_mass_total(const double* __restrict__ psum, const unsigned long long* __restrict__ pcnt, int nb,
                                  double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  unsigned long long u = 0;
  for (int b = 0; b < nb; ++b) {
    t += psum[b];
    u += pcnt[b];
  }
  out[0] = t;
  reinterpret_cast<unsigned long long*>(out)[1] = u;
}

// Largest key of the upper triangle (atomicMax on the bit patterns).
__global__ void __launch_bounds__(256) k_edge_maxkey(const double* __restrict__ E, int n,
                                                      unsigned long long* __restrict__ out) {
  unsigned long long m = 0;
  for (int i = blockIdx.x; i < n - 1; i += gridDim.x)
    for (int j = i + 1 + threadIdx.x; j < n; j += 256) m = max(m, dkey(E[(size_t)i * n + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Per row i: entries j > i with key > tau, and with key == tau.
__global__ void __launch_bounds__(256) k_edge_rowcount(const double* __restrict__ E, int n, unsigned long long tau,
                                                        int* __restrict__ cgt, int* __restrict__ ceq) {
  __shared__ int r1[8], r2[8];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    int a = 0, b = 0;
    for (int j = i + 1 + threadIdx.x; j < n; j += 256) {
      const unsigned long long kk = dkey(E[(size_t)i * n + j]);
      a += kk > tau;
      b += kk == tau;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      r1[threadIdx.x >> 5] = a;
      r2[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int x = 0, y = 0;
      for (int w = 0; w < 8; ++w) {
        x += r1[w];
        y += r2[w];
      }
      cgt[i] = x;
      ceq[i] = y;
    }
    __syncthreads();
  }
}

// Row offsets of the output (rows in order): row i writes its entries above
// tau and its ties with a global tie rank below c. One block.
__global__ void __launch_bounds__(1024) k_edge_offsets(const int* __restrict__ cgt, const int* __restrict__ ceq, int n,
                                                        long long c, long long* __restrict__ off,
                                                        long long* __restrict__ tie0, long long* __restrict__ total) {
  __shared__ long long ws[32], wt[32];
  __shared__ long long base, tbase;
  if (threadIdx.x == 0) base = tbase = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i0 = 0; i0 < n; i0 += 1024) {
    const int i = i0 + threadIdx.x;
    const long long eq = i < n ? ceq[i] : 0;
    // inclusive scan of ties, then of written counts
    long long t = eq;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane == 31) wt[w] = t;
    __syncthreads();
    long long tw = 0;
    for (int q = 0; q < w; ++q) tw += wt[q];
    const long long ties_before = tbase + tw + t - eq;
    const long long take = max(0LL, min(eq, c - ties_before));
    const long long cnt = (i < n ? cgt[i] : 0) + take;
    long long u = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += y;
    }
    if (lane == 31) ws[w] = u;
    __syncthreads();
    long long sw = 0;
    for (int q = 0; q < w; ++q) sw += ws[q];
    if (i < n) {
      off[i] = base + sw + u - cnt;
      tie0[i] = ties_before;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 0; q < 32; ++q) {
        base += ws[q];
        tbase += wt[q];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = base;
}

// Ordered write of the selected entries of each row: (i, j) pairs and values.
__global__ void __launch_bounds__(256) k_edge_write(const double* __restrict__ E, int n, unsigned long long tau,
                                                     long long c, const long long* __restrict__ off,
                                                     const long long* __restrict__ tie0, long long cap,
                                                     long long* __restrict__ ij, double* __restrict__ val) {
  __shared__ int wsel[8], wtie[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = blockIdx.x; i < n - 1; i += gridDim.x) {
    long long pos = off[i];
    long long tr = tie0[i];
    for (int j0 = i + 1; j0 < n; j0 += 256) {
      const int j = j0 + threadIdx.x;
      double v = 0.0;
      unsigned long long kk = 0;
      if (j < n) {
        v = E[(size_t)i * n + j];
        kk = dkey(v);
      }
      const bool tie = j < n && kk == tau;
      // tie rank within this chunk, then selection
      const unsigned bt = __ballot_sync(0xffffffffu, tie);
      if (lane == 0) wtie[w] = __popc(bt);
      __syncthreads();
      int tb = 0;
      for (int q = 0; q < w; ++q) tb += wtie[q];
      const long long my_tie = tr + tb + __popc(bt & ((1u << lane) - 1u));
      const bool sel = j < n && (kk > tau || (tie && my_tie < c));
      const unsigned bs = __ballot_sync(0xffffffffu, sel);
      if (lane == 0) wsel[w] = __popc(bs);
      __syncthreads();
      int sb = 0;
      for (int q = 0; q < w; ++q) sb += wsel[q];
      if (sel) {
        const long long p = pos + sb + __popc(bs & ((1u << lane) - 1u));
        if (p < cap) {
          ij[2 * p] = i;
          ij[2 * p + 1] = j;
          val[p] = v;
        }
      }
      int st = 0, tt = 0;
      for (int q = 0; q < 8; ++q) {
        st += wsel[q];
        tt += wtie[q];
      }
      pos += st;
      tr += tt;
      __syncthreads();
    }
  }
}

// The m largest edge scores of node nodes[b] (partners j != i; ties to the
// lower j), from the upper triangle: value (i, j) = E[min][max].
__global__ void __launch_bounds__(1024) k_node_top_edges(const double* __restrict__ E, int n,
                                                          const long long* __restrict__ nodes, int m,
                                                          long long* __restrict__ partner, double* __restrict__ pval) {
  __shared__ double sv[32];
  __shared__ int si[32];
  const int i = (int)nodes[blockIdx.x];
  double pv = INFINITY;
  int pi = -1;
  for (int t = 0; t < m; ++t) {
    double bv = -INFINITY;
    int bidx = INT_MAX;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      if (j == i) continue;
      const double v = i < j ? E[(size_t)i * n + j] : E[(size_t)j * n + i];
      const bool after = v < pv || (v == pv && j > pi);
      if (after && better(v, j, bv, bidx)) {
        bv = v;
        bidx = j;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (better(ov, oi, bv, bidx)) {
        bv = ov;
        bidx = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      sv[threadIdx.x >> 5] = bv;
      si[threadIdx.x >> 5] = bidx;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      bv = threadIdx.x < (blockDim.x >> 5) ? sv[threadIdx.x] : -INFINITY;
      bidx = threadIdx.x < (blockDim.x >> 5) ? si[threadIdx.x] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (better(ov, oi, bv, bidx)) {
          bv = ov;
          bidx = oi;
        }
      }
      if (threadIdx.x == 0) {
        sv[0] = bv;
        si[0] = bidx;
        partner[(size_t)blockIdx.x * m + t] = bidx == INT_MAX ? -1 : bidx;
        pval[(size_t)blockIdx.x * m + t] = bidx == INT_MAX ? 0.0 : bv;
      }
    }
    __syncthreads();
    pv = sv[0];
    pi = si[0];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- changed edges only
// Sec. 3.3: only node pairs whose weight changed (Delta A != 0) need their
// commute-time difference. When both graphs share sigma, A1 and A2 differ
// only in the rows and columns of the nodes whose series changed, so every
// edge score with a nonzero term has a changed endpoint: the pass below
// scores the m x n strip of those edges (the same per-edge arithmetic as the
// dense pass) and sums it per node.

// c2 - c1 for nodes c, j from the grid-split hi/lo planes (as in score_tile).
__device__ __forceinline__ double dc_pair_f32(const float* __restrict__ ah, const float* __restrict__ al,
                                              const float* __restrict__ bh, const float* __restrict__ bl, int n,
                                              int k, int c, int j) {
  float acc = 0.f, cmp = 0.f;
  for (int r = 0; r < k; ++r) {
    const size_t oc = (size_t)r * n + c, oj = (size_t)r * n + j;
    const float dah = __fsub_rn(ah[oc], ah[oj]);
    const float dal = __fsub_rn(al[oc], al[oj]);
    const float dbh = __fsub_rn(bh[oc], bh[oj]);
    const float dbl = __fsub_rn(bl[oc], bl[oj]);
    const float p = __fmul_rn(dah, dbh);
    float x = __fmaf_rn(dah, dbh, -p);
    x = __fmaf_rn(dah, dbl, x);
    x = __fmaf_rn(dal, dbh, x);
    const float t = __fadd_rn(acc, p);
    const float z = __fsub_rn(t, acc);
    const float err = __fadd_rn(__fsub_rn(acc, __fsub_rn(t, z)), __fsub_rn(p, z));
    acc = t;
    cmp = __fadd_rn(cmp, __fadd_rn(err, x));
  }
  return (double)acc + (double)cmp;
}

__device__ __forceinline__ double dc_pair_f64(const double* __restrict__ aT, const double* __restrict__ bT, int n,
                                              int k, int c, int j) {
  double acc = 0.0;
  for (int r = 0; r < k; ++r) {
    const size_t oc = (size_t)r * n + c, oj = (size_t)r * n + j;
    acc = fma(aT[oc] - aT[oj], bT[oc] - bT[oj], acc);
  }
  return acc;
}

// E[ci][j] = |A1_cj - A2_cj| |c2(c, j) - c1(c, j)| for changed node c = changed[ci].
__global__ void __launch_bounds__(256) k_changed_edges(const double* __restrict__ A1, const double* __restrict__ A2,
                                                        const void* __restrict__ ab, int n, int k, int fp64,
                                                        const int* __restrict__ changed, double* __restrict__ E) {
  const int ci = blockIdx.y;
  const int c = changed[ci];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double e = 0.0;
  if (j != c) {
    const size_t nk = (size_t)n * k;
    double dc;
    if (fp64) {
      const double* aT = static_cast<const double*>(ab);
      dc = dc_pair_f64(aT, aT + nk, n, k, c, j);
    } else {
      const float* ah = static_cast<const float*>(ab);
      dc = dc_pair_f32(ah, ah + nk, ah + 2 * nk, ah + 3 * nk, n, k, c, j);
    }
    const size_t o = (size_t)c * n + j;
    e = fabs(A1[o] - A2[o]) * fabs(dc);
  }
  E[(size_t)ci * n + j] = e;
}

// F_j = sum over changed c of E[c][j] (the terms of an unchanged node), in
// list order; changed nodes are overwritten by k_changed_rowsum.
__global__ void k_changed_colsum(const double* __restrict__ E, int m, int n, double* __restrict__ F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int ci = 0; ci < m; ++ci) s += E[(size_t)ci * n + j];
  F[j] = s;
}

// F_c = sum over j of E[c][j] for a changed node c (all of its terms).
__global__ void __launch_bounds__(256) k_changed_rowsum(const double* __restrict__ E, const int* __restrict__ changed,
                                                         int n, double* __restrict__ F) {
  __shared__ double red[8];
  const double* row = E + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += 256) s += row[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    F[changed[blockIdx.x]] = t;
  }
}

// Rows whose series differ (exact comparison): flag[i] = 1.
__global__ void k_row_differs(const double* __restrict__ X1, const double* __restrict__ X2, int n, int T,
                              int* __restrict__ flag) {
  const int i = blockIdx.x;
  bool d = false;
  for (int t = threadIdx.x; t < T; t += blockDim.x) d |= X1[(size_t)i * T + t] != X2[(size_t)i * T + t];
  d = __syncthreads_or(d);
  if (threadIdx.x == 0) flag[i] = d ? 1 : 0;
}

// Ordered compaction of the flagged rows (one block): list[count] = i.
__global__ void __launch_bounds__(1024) k_compact(const int* __restrict__ flag, int n, int* __restrict__ list,
                                                   int* __restrict__ count) {
  __shared__ int warp_sum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i0 = 0; i0 < n; i0 += 1024) {
    const int i = i0 + threadIdx.x;
    const int f = (i < n) ? flag[i] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_sum[w] = __popc(bal);
    __syncthreads();
    int off = 0;
    for (int q = 0; q < w; ++q) off += warp_sum[q];
    if (f) list[base + off + before] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int q = 0; q < 32; ++q) tot += warp_sum[q];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

// ---------------------------------------------------------------- batched form
// One launch per scoring step over all pairs of a batch; a block finds its
// pair (and block or tile) in a tile table.
__global__ void k_b_score_colmax(const uint32_t* __restrict__ tiles, const ScoreJob* __restrict__ jobs, int k) {
  const uint32_t t = tiles[blockIdx.x];
  const ScoreJob& J = jobs[t & 0xFFFu];
  score_colmax(J.Z1, J.Z2, J.vol1, J.vol2, J.n, k, J.cmax, (size_t)(t >> 12) * blockDim.x + threadIdx.x);
}

__global__ void k_b_score_prep(const uint32_t* __restrict__ tiles, const ScoreJob* __restrict__ jobs, int k, int fp64) {
  const uint32_t t = tiles[blockIdx.x];
  const ScoreJob& J = jobs[t & 0xFFFu];
  const size_t idx = (size_t)(t >> 12) * blockDim.x + threadIdx.x;
  const size_t nk = (size_t)J.n * k;
  if (fp64) {
    double* aT = static_cast<double*>(J.ab);
    score_prep64(J.Z1, J.Z2, J.vol1, J.vol2, J.n, k, aT, aT + nk, idx);
  } else {
    float* ah = static_cast<float*>(J.ab);
    score_prep(J.Z1, J.Z2, J.vol1, J.vol2, J.n, k, J.cmax, ah, ah + nk, ah + 2 * nk, ah + 3 * nk, idx);
  }
}

__global__ void __launch_bounds__(256) k_b_score_pairs(const uint32_t* __restrict__ tiles,
                                                        const ScoreJob* __restrict__ jobs, int k) {
  const uint32_t t = tiles[blockIdx.x];
  const ScoreJob& J = jobs[t & 0xFFFu];
  const size_t nk = (size_t)J.n * k;
  const float* ah = static_cast<const float*>(J.ab);
  score_tile(J.A1, J.A2, ah, ah + nk, ah + 2 * nk, ah + 3 * nk, J.n, k, J.contrib, (int)((t >> 12) & 0x3FFu),
             (int)(t >> 22));
}

__global__ void __launch_bounds__(256) k_b_score_pairs64(const uint32_t* __restrict__ tiles,
                                                          const ScoreJob* __restrict__ jobs, int k) {
  const uint32_t t = tiles[blockIdx.x];
  const ScoreJob& J = jobs[t & 0xFFFu];
  const size_t nk = (size_t)J.n * k;
  const double* aT = static_cast<const double*>(J.ab);
  score_tile64(J.A1, J.A2, aT, aT + nk, J.n, k, J.contrib, (int)((t >> 12) & 0x3FFu), (int)(t >> 22));
}

__global__ void k_b_score_reduce(const uint32_t* __restrict__ tiles, const ScoreJob* __restrict__ jobs) {
  const uint32_t t = tiles[blockIdx.x];
  const ScoreJob& J = jobs[t & 0xFFFu];
  const int i = (int)(t >> 12) * blockDim.x + threadIdx.x;
  if (i >= J.n) return;
  const int nb = (J.n + ST - 1) / ST;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += J.contrib[(size_t)b * J.n + i];
  J.F[i] = s;
}

__global__ void __launch_bounds__(1024) k_b_topk(const ScoreJob* __restrict__ jobs, int topk) {
  const ScoreJob& J = jobs[blockIdx.x];
  topk_block(J.F, J.n, topk, J.top);
}

}  // namespace

// a and b of both graphs in the layout the pair kernels read (float hi/lo
// planes on per-column grids, or float64), in the workspace buffer "score.ab".
int score_prepare(cdl_ctx* ctx, const double* Z1, const double* Z2, const double* vol1, const double* vol2, int n,
                  int k, bool fp64, void** vab) {
  cudaStream_t st = ctx->stream;
  const size_t nk = (size_t)n * k;
  CDL_TRY(ws_get(ctx, "score.ab", 16 * nk, vab));
  if (fp64) {
    double* aT = static_cast<double*>(*vab);
    Launch L(ctx, CDL_KC_MISC, 0);
    k_score_prep64<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(Z1, Z2, vol1, vol2, n, k, aT, aT + nk);
    return L.done();
  }
  float* ah = static_cast<float*>(*vab);
  void* vmax;
  CDL_TRY(ws_get(ctx, "score.cmax", 2 * (size_t)k * sizeof(unsigned), &vmax));
  unsigned* cmax = static_cast<unsigned*>(vmax);
  CDL_CUDA_TRY(cudaMemsetAsync(cmax, 0, 2 * (size_t)k * sizeof(unsigned), st));
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_score_colmax<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(Z1, Z2, vol1, vol2, n, k, cmax);
    CDL_TRY(L.done());
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_score_prep<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(Z1, Z2, vol1, vol2, n, k, cmax, ah, ah + nk,
                                                             ah + 2 * nk, ah + 3 * nk);
  return L.done();
}

namespace {
// The Z side of the tensor-core scores: column scales, the six slice planes
// of u / c and v / c, d_i in units of c^2 2^-48.
struct TcScorePrep {
  int rows = 0, k2p = 0;
  const void* u = nullptr;
  const void* v = nullptr;
  const long long* d = nullptr;
  const double* oscale = nullptr;
};

int tc_score_prepare(cdl_ctx* ctx, const double* Z1, const double* Z2, const double* vol1, const double* vol2, int n,
                     int k, TcScorePrep& q) {
  cudaStream_t st = ctx->stream;
  const int rows = (n + 127) / 128 * 128, k2p = (2 * k + 63) / 64 * 64;
  void *vcm, *vg, *vcs, *vu, *vv, *vd;
  CDL_TRY(ws_get(ctx, "score.tc.cmax", 2 * (size_t)k * sizeof(unsigned long long), &vcm));
  CDL_TRY(ws_get(ctx, "score.tc.g", (size_t)k * sizeof(double), &vg));
  CDL_TRY(ws_get(ctx, "score.tc.scale", 2 * sizeof(double), &vcs));
  CDL_TRY(ws_get(ctx, "score.tc.u", 6 * (size_t)rows * k2p * 2, &vu));
  CDL_TRY(ws_get(ctx, "score.tc.v", 6 * (size_t)rows * k2p * 2, &vv));
  CDL_TRY(ws_get(ctx, "score.tc.d", (size_t)rows * sizeof(long long), &vd));
  unsigned long long* cm = static_cast<unsigned long long*>(vcm);
  double* cs = static_cast<double*>(vcs);
  CDL_CUDA_TRY(cudaMemsetAsync(cm, 0, 2 * (size_t)k * sizeof(unsigned long long), st));
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_tcs_colmax<<<(unsigned)std::min(n, ctx->sm_count * 4), 256, 0, st>>>(Z1, Z2, vol1, vol2, n, k, cm);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_tcs_scales<<<1, 256, 0, st>>>(cm, k, static_cast<double*>(vg), cs);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    const size_t cnt = (size_t)rows * k2p;
    k_tcs_slice<<<(unsigned)std::min<size_t>((cnt + 255) / 256, (size_t)ctx->sm_count * 8), 256, 0, st>>>(
        Z1, Z2, vol1, vol2, n, k, rows, k2p, static_cast<const double*>(vg), cs, static_cast<__nv_bfloat16*>(vu),
        static_cast<__nv_bfloat16*>(vv));
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_tcs_diag<<<(rows + 7) / 8, 256, 0, st>>>(Z1, Z2, vol1, vol2, n, k, rows, cs, static_cast<long long*>(vd));
    CDL_TRY(L.done());
  }
  q.rows = rows;
  q.k2p = k2p;
  q.u = vu;
  q.v = vv;
  q.d = static_cast<const long long*>(vd);
  q.oscale = cs + 1;
  return CDL_OK;
}
}  // namespace

int cad_score_panels(cdl_ctx* ctx, const double* Z1, const double* Z2, const double* vol1, const double* vol2,
                     int64_t n64, int k, int P,
                     const std::function<int(int r0, int rows, const double** A1, const double** A2)>& fill, int topk,
                     double* F, int64_t* top_idx) {
  const int n = (int)n64;
  if (P % 128 || P <= 0) return CDL_ERR_INVALID_ARG;
  cudaStream_t st = ctx->stream;
  const int nb = (n + ST - 1) / ST;
  void* vc;
  CDL_TRY(ws_get(ctx, "score.contrib", (size_t)nb * n * sizeof(double), &vc));
  TcScorePrep q;
  CDL_TRY(tc_score_prepare(ctx, Z1, Z2, vol1, vol2, n, k, q));
  const long long nb64 = 2 * (q.rows / 128);
  auto off = [&](long long I) { return I * nb64 - I * (I - 1); };   // first upper tile of 128-row block I
  for (int r0 = 0; r0 < n; r0 += P) {
    const int rows = std::min(P, n - r0);
    const double *a1 = nullptr, *a2 = nullptr;
    CDL_TRY(fill(r0, rows, &a1, &a2));
    const long long I0 = r0 / 128, I1 = (r0 + rows + 127) / 128;
    CDL_TRY(score_tc_tiles(ctx, q.u, q.v, q.d, q.oscale, n, q.rows, q.k2p, a1, a2, r0, off(I0), off(I1),
                           static_cast<double*>(vc)));
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_score_reduce<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const double*>(vc), nb, n, F);
    CDL_TRY(L.done());
  }
  if (topk > 0) {
    Launch L(ctx, CDL_KC_TOPK, 0);
    k_topk<<<1, 1024, 0, st>>>(F, n, topk, top_idx);
    CDL_TRY(L.done());
  }
  return CDL_OK;
}

int cad_score(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1, const double* Z2,
              const double* vol1, const double* vol2, int64_t n64, int k, cdl_dtype score_dtype, int topk,
              double* F, int64_t* top_idx) {
  const int n = (int)n64;
  cudaStream_t st = ctx->stream;
  const int nb = (n + ST - 1) / ST;
  void *vab, *vc;
  const size_t nk = (size_t)n * k;
  const bool fp64 = score_dtype == CDL_F64;
  CDL_TRY(ws_get(ctx, "score.contrib", (size_t)nb * n * sizeof(double), &vc));
  if (score_dtype == CDL_BF16) {
    // Gram on the tensor cores from exact bf16 slices
    TcScorePrep q;
    CDL_TRY(tc_score_prepare(ctx, Z1, Z2, vol1, vol2, n, k, q));
    CDL_TRY(score_tc(ctx, q.u, q.v, q.d, q.oscale, n, q.rows, q.k2p, A1, A2, static_cast<double*>(vc)));
  } else {
  CDL_TRY(score_prepare(ctx, Z1, Z2, vol1, vol2, n, k, fp64, &vab));
  const long long tiles = (long long)nb * (nb + 1) / 2;
  if (fp64) {
    const double* aT = static_cast<const double*>(vab);
    Launch L(ctx, CDL_KC_SCORE, 8.0 * (double)n * (n - 1));
    k_score_pairs64<<<(unsigned)tiles, 256, 0, st>>>(A1, A2, aT, aT + nk, n, k, static_cast<double*>(vc));
    CDL_TRY(L.done());
  } else {
    const float* ah = static_cast<const float*>(vab);
    Launch L(ctx, CDL_KC_SCORE, 8.0 * (double)n * (n - 1));
    k_score_pairs<<<(unsigned)tiles, 256, 0, st>>>(A1, A2, ah, ah + nk, ah + 2 * nk, ah + 3 * nk, n, k,
                                                   static_cast<double*>(vc));
    CDL_TRY(L.done());
  }
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_score_reduce<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const double*>(vc), nb, n, F);
    CDL_TRY(L.done());
  }
  if (topk > 0) {
    Launch L(ctx, CDL_KC_TOPK, 0);
    k_topk<<<1, 1024, 0, st>>>(F, n, topk, top_idx);
    CDL_TRY(L.done());
  }
  return CDL_OK;
}

int cad_edges(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1, const double* Z2,
              const double* vol1, const double* vol2, int64_t n64, int k, bool fp64, double delta, int64_t cap,
              const int64_t* nodes, int n_nodes, int m, int64_t* ij, double* val, int64_t* partner, double* pval,
              double* F, cdl_edge_result* res) {
  const int n = (int)n64;
  cudaStream_t st = ctx->stream;
  const int nb = (n + ST - 1) / ST;
  void *vab, *vc, *vE, *vF, *vp, *vs, *vcnt, *voff;
  CDL_TRY(score_prepare(ctx, Z1, Z2, vol1, vol2, n, k, fp64, &vab));
  CDL_TRY(ws_get(ctx, "score.contrib", (size_t)nb * n * sizeof(double), &vc));
  CDL_TRY(ws_get(ctx, "edges.E", (size_t)n * n * sizeof(double), &vE));
  CDL_TRY(ws_get(ctx, "edges.F", (size_t)n * sizeof(double), &vF));
  const int mb = std::min(n, ctx->sm_count * 8);
  CDL_TRY(ws_get(ctx, "edges.part", (size_t)mb * 16, &vp));
  CDL_TRY(ws_get(ctx, "edges.scal", 64, &vs));
  CDL_TRY(ws_get(ctx, "edges.rowcnt", 2 * (size_t)n * sizeof(int), &vcnt));
  CDL_TRY(ws_get(ctx, "edges.rowoff", 2 * (size_t)n * sizeof(long long) + 16, &voff));
  double* E = static_cast<double*>(vE);
  double* Fw = F ? F : static_cast<double*>(vF);
  double* scal = static_cast<double*>(vs);
  double* psum = static_cast<double*>(vp);
  unsigned long long* pcnt = reinterpret_cast<unsigned long long*>(psum + mb);
  const long long tiles = (long long)nb * (nb + 1) / 2;
  {
    Launch L(ctx, CDL_KC_SCORE, 8.0 * (double)n * (n - 1));
    k_edge_pairs<<<(unsigned)tiles, 256, 0, st>>>(A1, A2, vab, n, k, fp64 ? 1 : 0, static_cast<double*>(vc), E);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_score_reduce<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const double*>(vc), nb, n, Fw);
    CDL_TRY(L.done());
  }
  // masses: total (tau = 0 counts every entry) and the largest key
  auto mass = [&](unsigned long long tau, double* sum, unsigned long long* cnt) -> int {
    {
      Launch L(ctx, CDL_KC_MISC, 0);
      k_edge_mass<<<mb, 256, 0, st>>>(E, n, tau, psum, pcnt);
      CDL_TRY(L.done());
    }
    {
      Launch L(ctx, CDL_KC_MISC, 0);
      k_edge_mass_total<<<1, 32, 0, st>>>(psum, pcnt, mb, scal);
      CDL_TRY(L.done());
    }
    double h[2];
    CDL_CUDA_TRY(cudaMemcpyAsync(h, scal, 16, cudaMemcpyDeviceToHost, st));
    CDL_CUDA_TRY(cudaStreamSynchronize(st));
    *sum = h[0];
    std::memcpy(cnt, &h[1], 8);
    return CDL_OK;
  };
  double total;
  unsigned long long m_all;
  CDL_TRY(mass(0ull, &total, &m_all));
  unsigned long long* dmax = reinterpret_cast<unsigned long long*>(scal + 4);
  CDL_CUDA_TRY(cudaMemsetAsync(dmax, 0, 8, st));
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_edge_maxkey<<<mb, 256, 0, st>>>(E, n, dmax);
    CDL_TRY(L.done());
  }
  unsigned long long kmax = 0;
  CDL_CUDA_TRY(cudaMemcpyAsync(&kmax, dmax, 8, cudaMemcpyDeviceToHost, st));
  CDL_CUDA_TRY(cudaStreamSynchronize(st));
  res->total = total;
  unsigned long long tau = 0;
  long long c = 0;
  bool none = total < delta;
  if (!none) {
    // largest tau in [0, kmax] with total - mass(>= tau) < delta (tau = 0 qualifies)
    unsigned long long lo = 0, hi = kmax;
    while (lo < hi) {
      const unsigned long long mid = lo + (hi - lo + 1) / 2;
      double s;
      unsigned long long cn;
      CDL_TRY(mass(mid, &s, &cn));
      if (total - s < delta)
        lo = mid;
      else
        hi = mid - 1;
    }
    tau = lo;
    // entries above tau are taken; ties at tau one by one in (i, j) order
    double s_gt = 0.0, s_ge = 0.0;
    unsigned long long c_gt = 0, c_ge = 0;
    CDL_TRY(mass(tau + 1, &s_gt, &c_gt));
    CDL_TRY(mass(tau, &s_ge, &c_ge));
    const long long ties = (long long)(c_ge - c_gt);
    double v;
    std::memcpy(&v, &tau, 8);
    double rem = total - s_gt;
    while (!(rem < delta) && c < ties) {
      rem -= v;
      ++c;
    }
    res->remaining = rem;
    res->threshold = v;
  } else {
    res->remaining = total;
    res->threshold = INFINITY;
    tau = ~0ull;   // nothing is above it
  }
  res->n_ties_taken = c;
  int* cgt = static_cast<int*>(vcnt);
  int* ceq = cgt + n;
  long long* off = static_cast<long long*>(voff);
  long long* tie0 = off + n;
  long long* tot = tie0 + n;
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_edge_rowcount<<<mb, 256, 0, st>>>(E, n, tau, cgt, ceq);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_edge_offsets<<<1, 1024, 0, st>>>(cgt, ceq, n, none ? 0 : c, off, tie0, tot);
    CDL_TRY(L.done());
  }
  if (cap > 0) {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_edge_write<<<mb, 256, 0, st>>>(E, n, tau, none ? 0 : c, off, tie0, cap, reinterpret_cast<long long*>(ij), val);
    CDL_TRY(L.done());
  }
  if (n_nodes > 0 && m > 0) {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_node_top_edges<<<n_nodes, 1024, 0, st>>>(E, n, reinterpret_cast<const long long*>(nodes), m,
                                               reinterpret_cast<long long*>(partner), pval);
    CDL_TRY(L.done());
  }
  long long count = 0;
  CDL_CUDA_TRY(cudaMemcpyAsync(&count, tot, 8, cudaMemcpyDeviceToHost, st));
  CDL_CUDA_TRY(cudaStreamSynchronize(st));
  res->n_edges = count;
  return CDL_OK;
}

int changed_nodes(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n, int T, int* list, int* count_dev) {
  void* vf;
  CDL_TRY(ws_get(ctx, "score.changed_flag", (size_t)n * sizeof(int), &vf));
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_row_differs<<<(unsigned)n, 128, 0, ctx->stream>>>(X1, X2, (int)n, T, static_cast<int*>(vf));
    CDL_TRY(L.done());
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_compact<<<1, 1024, 0, ctx->stream>>>(static_cast<const int*>(vf), (int)n, list, count_dev);
  return L.done();
}

int cad_score_changed(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1, const double* Z2,
                      const double* vol1, const double* vol2, int64_t n64, int k, bool fp64, const int* changed,
                      int m, int topk, double* F, int64_t* top_idx) {
  const int n = (int)n64;
  cudaStream_t st = ctx->stream;
  void *vab, *vE;
  CDL_TRY(score_prepare(ctx, Z1, Z2, vol1, vol2, n, k, fp64, &vab));
  if (m > 0) {
    CDL_TRY(ws_get(ctx, "score.changed_E", (size_t)m * n * sizeof(double), &vE));
    double* E = static_cast<double*>(vE);
    {
      dim3 g((n + 255) / 256, m);
      Launch L(ctx, CDL_KC_SCORE, 16.0 * (double)m * n);
      k_changed_edges<<<g, 256, 0, st>>>(A1, A2, vab, n, k, fp64 ? 1 : 0, changed, E);
      CDL_TRY(L.done());
    }
    {
      Launch L(ctx, CDL_KC_MISC, 0);
      k_changed_colsum<<<(n + 255) / 256, 256, 0, st>>>(E, m, n, F);
      CDL_TRY(L.done());
    }
    Launch L(ctx, CDL_KC_MISC, 0);
    k_changed_rowsum<<<m, 256, 0, st>>>(E, changed, n, F);
    CDL_TRY(L.done());
  } else {
    CDL_CUDA_TRY(cudaMemsetAsync(F, 0, (size_t)n * sizeof(double), st));
  }
  if (topk > 0) {
    Launch L(ctx, CDL_KC_TOPK, 0);
    k_topk<<<1, 1024, 0, st>>>(F, n, topk, top_idx);
    CDL_TRY(L.done());
  }
  return CDL_OK;
}

int cad_score_grouped(cdl_ctx* ctx, const ScoreJob* jobs, int G, int k, bool fp64, int topk, BTiles elem,
                      BTiles pairs, BTiles nodes, double bytes, unsigned* cmax_all) {
  cudaStream_t st = ctx->stream;
  if (!fp64) {
    CDL_CUDA_TRY(cudaMemsetAsync(cmax_all, 0, (size_t)G * 2 * k * sizeof(unsigned), st));
    Launch L(ctx, CDL_KC_MISC, 0);
    k_b_score_colmax<<<elem.count, 256, 0, st>>>(elem.p, jobs, k);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_b_score_prep<<<elem.count, 256, 0, st>>>(elem.p, jobs, k, fp64 ? 1 : 0);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_SCORE, bytes);
    if (fp64)
      k_b_score_pairs64<<<pairs.count, 256, 0, st>>>(pairs.p, jobs, k);
    else
      k_b_score_pairs<<<pairs.count, 256, 0, st>>>(pairs.p, jobs, k);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_b_score_reduce<<<nodes.count, 256, 0, st>>>(nodes.p, jobs);
    CDL_TRY(L.done());
  }
  if (topk > 0) {
    Launch L(ctx, CDL_KC_TOPK, 0);
    k_b_topk<<<G, 1024, 0, st>>>(jobs, topk);
    CDL_TRY(L.done());
  }
  return CDL_OK;
}

}  // namespace cdl
