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
#include <cfloat>
#include <climits>
#include <cmath>

#include "internal.h"

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

__device__ __forceinline__ void tri_index(int t, int nb, int& bi, int& bj) {
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

// Per-tile accumulation of |A1 - A2| |c2 - c1| into row and column partials.
__device__ __forceinline__ void tile_finish(const double* __restrict__ A1, const double* __restrict__ A2,
                                            int n, int i0, int j0, int bi, int bj, int tx, int ty,
                                            const double (&dc)[4][4], double* __restrict__ contrib,
                                            double (*rsum)[17], double (*csum)[17]) {
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
                                           double* __restrict__ contrib, int bi, int bj) {
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
  tile_finish(A1, A2, n, i0, j0, bi, bj, tx, ty, dc, contrib, rsum, csum);
}

__global__ void __launch_bounds__(256) k_score_pairs(const double* __restrict__ A1, const double* __restrict__ A2,
                                                      const float* __restrict__ ah, const float* __restrict__ al,
                                                      const float* __restrict__ bh, const float* __restrict__ bl,
                                                      int n, int k, double* __restrict__ contrib) {
  const int nb = (n + ST - 1) / ST;
  int bi, bj;
  tri_index(blockIdx.x, nb, bi, bj);
  score_tile(A1, A2, ah, al, bh, bl, n, k, contrib, bi, bj);
}

// float64 variant: c2 - c1 = sum_r (a_ir - a_jr)(b_ir - b_jr) in float64.
__device__ __forceinline__ void score_tile64(const double* __restrict__ A1, const double* __restrict__ A2,
                                             const double* __restrict__ aT, const double* __restrict__ bT, int n,
                                             int k, double* __restrict__ contrib, int bi, int bj) {
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
  tile_finish(A1, A2, n, i0, j0, bi, bj, tx, ty, acc, contrib, rsum, csum);
}

__global__ void __launch_bounds__(256) k_score_pairs64(const double* __restrict__ A1,
                                                        const double* __restrict__ A2,
                                                        const double* __restrict__ aT,
                                                        const double* __restrict__ bT, int n, int k,
                                                        double* __restrict__ contrib) {
  const int nb = (n + ST - 1) / ST;
  int bi, bj;
  tri_index(blockIdx.x, nb, bi, bj);
  score_tile64(A1, A2, aT, bT, n, k, contrib, bi, bj);
}


__global__ void k_score_reduce(const double* __restrict__ contrib, int nb, int n, double* __restrict__ F) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += contrib[(size_t)b * n + i];
  F[i] = s;
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

int cad_score(cdl_ctx* ctx, const double* A1, const double* A2, const double* Z1, const double* Z2,
              const double* vol1, const double* vol2, int64_t n64, int k, bool fp64, int topk,
              double* F, int64_t* top_idx) {
  const int n = (int)n64;
  cudaStream_t st = ctx->stream;
  const int nb = (n + ST - 1) / ST;
  void *vab, *vc;
  const size_t nk = (size_t)n * k;
  CDL_TRY(score_prepare(ctx, Z1, Z2, vol1, vol2, n, k, fp64, &vab));
  CDL_TRY(ws_get(ctx, "score.contrib", (size_t)nb * n * sizeof(double), &vc));
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
