// Graph build (Sec. 2; kernel of Sec. 4.2.1; D = A 1 of Sec. 3.2):
//   1. squared distances ||x_i - x_j||^2 for all pairs (upper-triangle tiles,
//      mirrored), exact in int64 when X lies on the 2^-16 grid, otherwise in
//      float64 with one rounding per subtraction, product and sum;
//   2. sigma = lower median of the distances over i < j by an exact radix
//      select on the float64 bit patterns (distances are >= 0, so their bit
//      patterns order like the values);
//   3. A_ij = exp(-d2_ij / (2 sigma^2)), A_ii = 0, D_i = sum_j A_ij, vol.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include <cuda_bf16.h>

#include "ff.cuh"

#include "internal.h"
#include "tiles.cuh"

namespace cdl {
namespace {

constexpr int DT = 64;          // distance tile (rows and columns)
constexpr int DTK = 32;         // samples per smem chunk
constexpr int RADIX_BITS = 12;
constexpr int RADIX_BINS = 1 << RADIX_BITS;

struct SelectState {
  unsigned long long prefix;    // selected high bits so far
  unsigned long long mask;      // which bits are selected
  long long rank;               // rank within the still-matching keys
  int flags;                    // bit 0: input off the 2^-16 grid
  int pad;
  unsigned long long ncomp;     // keys matching the prefix of the first two digits
};
// The third pass of the single-graph select also copies the keys that match
// the first two digits (about 2^-12 of the value range around the median) to
// a buffer of min(SELECT_CAP, max(m / 64, 1024)) keys (m keys in all); the
// last three passes then read that buffer instead of the whole triangle,
// unless more keys matched than it holds.
constexpr long long SELECT_CAP = 1ll << 22;
static_assert(sizeof(SelectState) <= 64, "the batched form keeps 64 bytes for the state");

// X (float64, n x T) -> int32 fixed point a = x * 2^16, stored transposed
// (T x n) for coalesced tile loads; flags input off the grid.
__global__ void k_to_fixed(const double* __restrict__ X, int* __restrict__ Xt, int n, int T,
                           SelectState* st) {
  const size_t total = (size_t)n * T;
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  bool off = false;
  for (; idx < total; idx += stride) {
    double a = X[idx] * 65536.0;   // exact scaling by a power of two
    bool ok = (a == rint(a)) && fabs(a) < 8388608.0;
    off |= !ok;
    size_t i = idx / T, t = idx % T;
    Xt[t * n + i] = ok ? (int)a : 0;
  }
  if (__syncthreads_or(off) && threadIdx.x == 0) atomicOr(&st->flags, 1);
}

// Three signed base-256 digit planes of a = x 2^16 for the tensor-core
// distances (rows x tp bf16 each, zero padded): a = d0 + 2^8 d1 + 2^16 d2 with
// |d| <= 128, exact in bf16. Inputs off the grid give zeros (the float64
// kernel handles them).
__global__ void __launch_bounds__(256) k_slice_x(const double* __restrict__ X, int n, int T, int rows, int tp,
                                                  __nv_bfloat16* __restrict__ planes) {
  const size_t plane = (size_t)rows * tp;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / tp), t = (int)(idx % tp);
    int a = 0;
    if (i < n && t < T) {
      const double v = X[(size_t)i * T + t] * 65536.0;
      if (v == rint(v) && fabs(v) < 8388608.0) a = (int)v;
    }
    const int d0 = ((a + 128) & 255) - 128;
    const int a1 = (a - d0) >> 8;                         // exact: a - d0 is a multiple of 256
    const int d1 = ((a1 + 128) & 255) - 128;
    const int d2 = (a1 - d1) >> 8;
    planes[idx] = __int2bfloat16_rn(d0);
    planes[plane + idx] = __int2bfloat16_rn(d1);
    planes[2 * plane + idx] = __int2bfloat16_rn(d2);
  }
}

// |a_i|^2 = sum_t a_it^2 in int64 (exact), one warp per row; padded rows 0.
__global__ void __launch_bounds__(256) k_row_norms(const double* __restrict__ X, int n, int T, int rows,
                                                    long long* __restrict__ norms) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= rows) return;
  long long acc = 0;
  if (row < n)
    for (int t = lane; t < T; t += 32) {
      const double v = X[(size_t)row * T + t] * 65536.0;
      const long long a = (v == rint(v) && fabs(v) < 8388608.0) ? (long long)v : 0;
      acc += a * a;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) norms[row] = acc;
}


// Exact squared distances on the 2^-16 grid: int64 sums of squared int32
// differences, written as float64 multiples of 2^-32 to both (i,j) and (j,i).
__device__ __forceinline__ void dist_int_tile(const int* __restrict__ Xt, int n, int T, double* __restrict__ A,
                                              int bi, int bj) {
  __shared__ __align__(16) int As[DTK][DT];
  __shared__ __align__(16) int Bs[DTK][DT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = bi * DT, c0 = bj * DT;
  long long acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0;
  for (int t0 = 0; t0 < T; t0 += DTK) {
    // load 32 samples x 64 nodes of each side from the transposed copy
    for (int e = threadIdx.x; e < DT * DTK; e += 256) {
      int row = e % DT, tt = e / DT;
      int ia = r0 + row, ib = c0 + row, t = t0 + tt;
      As[tt][row] = (ia < n && t < T) ? Xt[(size_t)t * n + ia] : 0;
      Bs[tt][row] = (ib < n && t < T) ? Xt[(size_t)t * n + ib] : 0;
    }
    __syncthreads();
#pragma unroll 4
    for (int tt = 0; tt < DTK; ++tt) {
      int4 a = *reinterpret_cast<const int4*>(&As[tt][ty * 4]);
      int4 b = *reinterpret_cast<const int4*>(&Bs[tt][tx * 4]);
      int av[4] = {a.x, a.y, a.z, a.w};
      int bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          int dd = av[u] - bv[v];
          acc[u][v] += (long long)dd * dd;
        }
    }
    __syncthreads();
  }
  const double q = 1.0 / 4294967296.0;   // 2^-32
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int i = r0 + ty * 4 + u;
    if (i >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int j = c0 + tx * 4 + v;
      if (j >= n) continue;
      double d2 = (double)acc[u][v] * q;
      A[(size_t)i * n + j] = d2;
      if (bi != bj) A[(size_t)j * n + i] = d2;
    }
  }
}

__global__ void __launch_bounds__(256) k_dist_int(const int* __restrict__ Xt, int n, int T,
                                                   double* __restrict__ A, const SelectState* st) {
  if (st->flags & 1) return;   // off-grid input: the float64 kernel handles it
  const int nb = (n + DT - 1) / DT;
  int bi, bj;
  block_tri_index(nb, bi, bj);
  dist_int_tile(Xt, n, T, A, bi, bj);
}

// Float64 squared distances for inputs off the grid: same tiling, samples in
// ascending order, explicit round-to-nearest operations (no contraction).
__device__ __forceinline__ void dist_f64_tile(const double* __restrict__ X, int n, int T, double* __restrict__ A,
                                              int bi, int bj) {
  __shared__ double As[DTK][DT + 1];
  __shared__ double Bs[DTK][DT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = bi * DT, c0 = bj * DT;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int t0 = 0; t0 < T; t0 += DTK) {
    for (int e = threadIdx.x; e < DT * DTK; e += 256) {
      int row = e / DTK, tt = e % DTK;
      int ia = r0 + row, ib = c0 + row, t = t0 + tt;
      As[tt][row] = (ia < n && t < T) ? X[(size_t)ia * T + t] : 0.0;
      Bs[tt][row] = (ib < n && t < T) ? X[(size_t)ib * T + t] : 0.0;
    }
    __syncthreads();
    const int tmax = min(DTK, T - t0);
    for (int tt = 0; tt < tmax; ++tt) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double dd = __dsub_rn(As[tt][ty * 4 + u], Bs[tt][tx * 4 + v]);
          acc[u][v] = __dadd_rn(acc[u][v], __dmul_rn(dd, dd));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int i = r0 + ty * 4 + u;
    if (i >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int j = c0 + tx * 4 + v;
      if (j >= n) continue;
      A[(size_t)i * n + j] = acc[u][v];
      if (bi != bj) A[(size_t)j * n + i] = acc[u][v];
    }
  }
}

__global__ void __launch_bounds__(256) k_dist_f64(const double* __restrict__ X, int n, int T,
                                                   double* __restrict__ A, const SelectState* st) {
  if (!(st->flags & 1)) return;
  const int nb = (n + DT - 1) / DT;
  int bi, bj;
  block_tri_index(nb, bi, bj);
  dist_f64_tile(X, n, T, A, bi, bj);
}

__global__ void k_select_init(SelectState* st, long long rank) {
  st->prefix = 0;
  st->mask = 0;
  st->rank = rank;
  st->flags = 0;
  st->ncomp = 0;
}

// Histogram of the `bits`-wide digit at `shift` over keys of the upper
// triangle matching the current prefix.
// rows r0, r0 + rstep, ... < r1 of the upper triangle
// (A holds rows roff .. : row i at A + (i - roff) n)
__device__ __forceinline__ void select_hist_rows(const double* __restrict__ A, int n, int shift, int bits,
                                                 const SelectState* __restrict__ st,
                                                 unsigned long long* __restrict__ hist, int r0, int r1, int rstep,
                                                 int roff = 0) {
  __shared__ unsigned int h[RADIX_BINS];
  for (int b = threadIdx.x; b < RADIX_BINS; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const unsigned long long prefix = st->prefix, mask = st->mask;
  const unsigned long long dmask = (1ull << bits) - 1ull;
  const unsigned long long* K = reinterpret_cast<const unsigned long long*>(A);
  for (int i = r0; i < r1; i += rstep) {
    const unsigned long long* row = K + (size_t)(i - roff) * n;
    for (int j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
      unsigned long long key = row[j];
      if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & dmask], 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < RADIX_BINS; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], (unsigned long long)h[b]);
}

__global__ void __launch_bounds__(512) k_select_hist(const double* __restrict__ A, int n, int shift,
                                                      int bits, const SelectState* __restrict__ st,
                                                      unsigned long long* __restrict__ hist) {
  select_hist_rows(A, n, shift, bits, st, hist, blockIdx.x, n - 1, gridDim.x);
}

// The same histogram over rows r0 .. r1 - 1 of a panel holding rows r0 ..
__global__ void __launch_bounds__(512) k_select_hist_panel(const double* __restrict__ P, int n, int shift, int bits,
                                                            const SelectState* __restrict__ st,
                                                            unsigned long long* __restrict__ hist, int r0, int r1) {
  select_hist_rows(P, n, shift, bits, st, hist, r0 + blockIdx.x, r1, gridDim.x, r0);
}

// The third pass: the histogram of select_hist_rows, and every key matching
// the current prefix appended to buf (the first `cap`; st->ncomp counts all).
__global__ void __launch_bounds__(512) k_select_hist_compact(const double* __restrict__ A, int n, int shift, int bits,
                                                              SelectState* st, unsigned long long* __restrict__ hist,
                                                              unsigned long long* __restrict__ buf, long long cap) {
  __shared__ unsigned int h[RADIX_BINS];
  for (int b = threadIdx.x; b < RADIX_BINS; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const unsigned long long prefix = st->prefix, mask = st->mask;
  const unsigned long long dmask = (1ull << bits) - 1ull;
  const unsigned long long* K = reinterpret_cast<const unsigned long long*>(A);
  for (int i = blockIdx.x; i < n - 1; i += gridDim.x) {
    const unsigned long long* row = K + (size_t)i * n;
    for (int j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
      const unsigned long long key = row[j];
      if ((key & mask) == prefix) {
        atomicAdd(&h[(key >> shift) & dmask], 1u);
        const unsigned long long pos = atomicAdd(&st->ncomp, 1ull);
        if (pos < (unsigned long long)cap) buf[pos] = key;
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < RADIX_BINS; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], (unsigned long long)h[b]);
}

// The later passes: the histogram over the copied keys, or over the whole
// triangle when they did not fit.
__global__ void __launch_bounds__(512) k_select_hist_buf(const double* __restrict__ A, int n, int shift, int bits,
                                                          const SelectState* __restrict__ st,
                                                          unsigned long long* __restrict__ hist,
                                                          const unsigned long long* __restrict__ buf, long long cap) {
  const unsigned long long nc = st->ncomp;
  if (nc > (unsigned long long)cap) {
    select_hist_rows(A, n, shift, bits, st, hist, blockIdx.x, n - 1, gridDim.x);
    return;
  }
  __shared__ unsigned int h[RADIX_BINS];
  for (int b = threadIdx.x; b < RADIX_BINS; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const unsigned long long prefix = st->prefix, mask = st->mask;
  const unsigned long long dmask = (1ull << bits) - 1ull;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nc; q += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long key = buf[q];
    if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & dmask], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < RADIX_BINS; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], (unsigned long long)h[b]);
}

// Pick the bin holding the remaining rank; extend the prefix; clear hist.
__device__ __forceinline__ void select_step(SelectState* st, unsigned long long* hist, int shift, int bits,
                                            double* sigma_out, int last) {
  __shared__ unsigned long long cnt[RADIX_BINS];
  const int nbins = 1 << bits;
  for (int b = threadIdx.x; b < RADIX_BINS; b += blockDim.x) {
    cnt[b] = hist[b];
    hist[b] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long r = st->rank;
    int b = 0;
    for (; b < nbins; ++b) {
      if ((long long)cnt[b] > r) break;
      r -= (long long)cnt[b];
    }
    if (b >= nbins) b = nbins - 1;   // unreachable for a consistent histogram
    unsigned long long dm = (unsigned long long)(nbins - 1) << shift;
    st->prefix |= (unsigned long long)b << shift;
    st->mask |= dm;
    st->rank = r;
    if (last) {
      double d2 = __longlong_as_double((long long)st->prefix);
      *sigma_out = sqrt(d2);
    }
  }
}

__global__ void k_select_step(SelectState* st, unsigned long long* hist, int shift, int bits,
                              double* sigma_out, int last) {
  select_step(st, hist, shift, bits, sigma_out, last);
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// A_ij = exp(-d2_ij / (2 sigma^2)) (KERN = KERNEL_GAUSSIAN) or
// A_ij = exp(-sqrt(d2_ij) / sigma) (KERN = KERNEL_EXP, the synthetic-data
// kernel of Sec. 4.2.1), A_ii = 0, D_i = row sum. One block per row.
// The exponential is ff_exp_neg_prod: the argument d2 * (1 / (2 sigma^2)), or
// sqrt(d2) (sqrt_nonneg: within one ulp) times 1 / sigma, is formed exactly in
// 128-bit integers and reduced there (by k ln2, then by j / 32 through a
// per-block table), then a float-float series (about 1.4e-14 relative) and an
// integer assembly of the float64 result: no float64
// operation but the three of the exp kernel's square root, float64 being the
// scarce pipe. The row sum is accumulated in float-float (terms below 2^-100 are
// dropped from the sum, not from A).
enum { KERNEL_GAUSSIAN = 0, KERNEL_EXP = 1 };

template <int KERN = KERNEL_GAUSSIAN>
__device__ __forceinline__ void kernel_row(double* __restrict__ A, int n, double rcp, double* __restrict__ D,
                                           int i, const ff* __restrict__ tab, int roff = 0) {
  __shared__ double red[8];
  {
    double* row = A + (size_t)(i - roff) * n;
    const float rcpf = d2f_trunc(rcp);
    ff acc = {0.f, 0.f};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double x = KERN == KERNEL_EXP ? sqrt_nonneg(row[j]) : row[j];
      double a = 0.0;
      if (j != i) {
        if (__fmul_rn(d2f_trunc(x), rcpf) < 680.f) {          // t = x rcp well below 690
          int k;
          const ff q = ff_exp_neg_prod(x, rcp, k, tab);
          a = ff_scaled_to_double(q, k);
          if (k <= 100) {
            const float sc = __int_as_float((127 - k) << 23);   // 2^-k
            const ff ts = two_sum(acc.hi, __fmul_rn(q.hi, sc));
            acc.hi = ts.hi;
            acc.lo = __fadd_rn(acc.lo, __fadd_rn(ts.lo, __fmul_rn(q.lo, sc)));
          }
        } else {
          a = exp(-(x * rcp));
        }
      }
      row[j] = a;
    }
    double accd = (double)acc.hi + (double)acc.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) accd += __shfl_xor_sync(0xffffffffu, accd, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = accd;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      D[i] = t;
    }
    __syncthreads();
  }
}

template <int KERN = KERNEL_GAUSSIAN>
__global__ void __launch_bounds__(256) k_kernel_rows(double* __restrict__ A, int n,
                                                      const double* __restrict__ sigma,
                                                      double* __restrict__ D) {
  const double s = *sigma;
  const double rcp = KERN == KERNEL_EXP ? 1.0 / s : 1.0 / (2.0 * (s * s));
  __shared__ ff tab[FF_EXP_TABLE];
  ff_exp_table(tab);
  __syncthreads();
  for (int i = blockIdx.x; i < n; i += gridDim.x) kernel_row<KERN>(A, n, rcp, D, i, tab);
}

// Rows r0 .. r1 - 1 of a panel holding rows r0 .. (squared distances in,
// kernel values out), their degrees into D[i].
__global__ void __launch_bounds__(256) k_kernel_rows_panel(double* __restrict__ P, int n,
                                                            const double* __restrict__ sigma, double* __restrict__ D,
                                                            int r0, int r1) {
  const double s = *sigma;
  const double rcp = 1.0 / (2.0 * (s * s));
  __shared__ ff tab[FF_EXP_TABLE];
  ff_exp_table(tab);
  __syncthreads();
  for (int i = r0 + blockIdx.x; i < r1; i += gridDim.x) kernel_row<KERNEL_GAUSSIAN>(P, n, rcp, D, i, tab, r0);
}

// Kernel values over the upper block triangle of 64 x 64 tiles (A is
// symmetric, so half the exponentials of the row-by-row pass): a block
// evaluates tile (bi, bj), bj >= bi (a diagonal tile all of its entries),
// writes it and, off the diagonal, its mirror through shared memory (both
// writes coalesced), and leaves the tile's row and column sums of A
// (float-float, the entries split with integer operations) in the slots of
// the 64-node partner blocks: part[bj][i] for its rows, part[bi][j] for its
// columns (rows only on the diagonal). D_i is the fixed-order sum of node i's
// slots (k_part_sums). Same entry arithmetic as kernel_row.
template <int KERN>
__global__ void __launch_bounds__(256) k_kernel_tiles(double* __restrict__ A, int n, const double* __restrict__ sigma,
                                                       double* __restrict__ part, unsigned long long* __restrict__ amax) {
  __shared__ double tt[DT][DT + 1];                     // tt[c][r] = A(i0 + r, j0 + c)
  __shared__ unsigned long long wmax[8];
  const int nb = (n + DT - 1) / DT;
  __shared__ double rcp_s;                               // float64 division and square root once per block
  __shared__ int tile_s[2];
  __shared__ ff tab[FF_EXP_TABLE];
  ff_exp_table(tab);
  if (threadIdx.x == 0) {
    tri_index(blockIdx.x, nb, tile_s[0], tile_s[1]);
    const double sg = *sigma;
    rcp_s = KERN == KERNEL_EXP ? 1.0 / sg : 1.0 / (2.0 * (sg * sg));
  }
  __syncthreads();
  const int bi = tile_s[0], bj = tile_s[1];
  const int i0 = bi * DT, j0 = bj * DT;
  const double rcp = rcp_s;
  const float rcpf = d2f_trunc(rcp);
  const int c = threadIdx.x & (DT - 1), rg = threadIdx.x >> 6;
#pragma unroll 4
  for (int m = 0; m < DT / 4; ++m) {
    const int r = rg + 4 * m, i = i0 + r, j = j0 + c;
    double a = 0.0;
    if (i < n && j < n) {
      double* pa = A + (size_t)i * n + j;
      if (i != j) {
        const double x = KERN == KERNEL_EXP ? sqrt_nonneg(*pa) : *pa;
        if (__fmul_rn(d2f_trunc(x), rcpf) < 680.f) {
          int k;
          const ff q = ff_exp_neg_prod(x, rcp, k, tab);
          a = ff_scaled_to_double(q, k);
        } else {
          a = exp(-(x * rcp));
        }
      }
      *pa = a;
    }
    tt[c][r] = a;
  }
  if (amax) {                                            // max A (a >= 0: bit patterns order like values)
    unsigned long long mb = 0;
#pragma unroll 4
    for (int m = 0; m < DT / 4; ++m) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(tt[c][rg + 4 * m]);
      mb = b > mb ? b : mb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = v > mb ? v : mb;
    }
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mb;
  }
  __syncthreads();
  if (amax && threadIdx.x == 0) {
    unsigned long long mb = wmax[0];
    for (int w = 1; w < 8; ++w) mb = wmax[w] > mb ? wmax[w] : mb;
    if (mb) atomicMax(amax, mb);
  }
  if (bi != bj) {                                        // mirror: lanes write consecutive columns of row j
#pragma unroll 4
    for (int m = 0; m < DT / 4; ++m) {
      const int cc = rg + 4 * m, r = threadIdx.x & (DT - 1);
      const int j = j0 + cc, i = i0 + r;
      if (j < n && i < n) A[(size_t)j * n + i] = tt[cc][r];
    }
  }
  if (threadIdx.x < DT) {                                // row sums of the tile
    const int r = threadIdx.x, i = i0 + r;
    ff acc = {0.f, 0.f};
    for (int cc = 0; cc < DT; ++cc) acc = ff_add(acc, split_nonneg(tt[cc][r]));
    if (i < n) part[(size_t)bj * n + i] = (double)acc.hi + (double)acc.lo;
  } else if (threadIdx.x < 2 * DT && bi != bj) {         // column sums (the mirror's row sums)
    const int cc = threadIdx.x - DT, j = j0 + cc;
    ff acc = {0.f, 0.f};
    for (int r = 0; r < DT; ++r) acc = ff_add(acc, split_nonneg(tt[cc][r]));
    if (j < n) part[(size_t)bi * n + j] = (double)acc.hi + (double)acc.lo;
  }
}

__global__ void k_part_sums(const double* __restrict__ part, int nb, int n, double* __restrict__ D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(size_t)b * n + i];
  D[i] = s;
}

// vol = sum_i D_i (single block, fixed order per thread then tree).
__device__ __forceinline__ void block_sum_to(const double* __restrict__ v, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
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

__global__ void k_sum(const double* __restrict__ v, int n, double* __restrict__ out) { block_sum_to(v, n, out); }

// ---------------------------------------------------------------- batched form
// The same steps for every graph of a batch, one launch per step; a block
// finds its graph and work item in a tile table.
__global__ void k_g_select_init(const GGraph* __restrict__ gs) {
  const GGraph& G = gs[blockIdx.x];
  SelectState* st = static_cast<SelectState*>(G.sel);
  const long long m = (long long)G.n * (G.n - 1) / 2;
  st->prefix = 0;
  st->mask = 0;
  st->rank = (m - 1) / 2;
  st->flags = 0;
  st->ncomp = 0;
}

__global__ void k_g_to_fixed(const uint32_t* __restrict__ tiles, const GGraph* __restrict__ gs) {
  const uint32_t t = tiles[blockIdx.x];
  const GGraph& G = gs[t & 0xFFFu];
  const size_t total = (size_t)G.n * G.T;
  const size_t base = (size_t)(t >> 12) * 1024;
  bool off = false;
  for (size_t idx = base + threadIdx.x; idx < total && idx < base + 1024; idx += blockDim.x) {
    const double a = G.X[idx] * 65536.0;
    const bool ok = (a == rint(a)) && fabs(a) < 8388608.0;
    off |= !ok;
    const size_t i = idx / G.T, tt = idx % G.T;
    G.Xt[tt * G.n + i] = ok ? (int)a : 0;
  }
  if (__syncthreads_or(off) && threadIdx.x == 0) atomicOr(&static_cast<SelectState*>(G.sel)->flags, 1);
}

// tiles: g | bi << 12 | bj << 22 (64-node blocks, bi <= bj)
__global__ void __launch_bounds__(256) k_g_dist(const uint32_t* __restrict__ tiles, const GGraph* __restrict__ gs) {
  const uint32_t t = tiles[blockIdx.x];
  const GGraph& G = gs[t & 0xFFFu];
  const int bi = (int)((t >> 12) & 0x3FFu), bj = (int)(t >> 22);
  if (static_cast<const SelectState*>(G.sel)->flags & 1)
    dist_f64_tile(G.X, G.n, G.T, G.A, bi, bj);
  else
    dist_int_tile(G.Xt, G.n, G.T, G.A, bi, bj);
}

__global__ void __launch_bounds__(512) k_g_select_hist(const int4* __restrict__ tiles, const GGraph* __restrict__ gs,
                                                        int shift, int bits) {
  const int4 t = tiles[blockIdx.x];
  const GGraph& G = gs[t.x];
  SelectState* st = static_cast<SelectState*>(G.sel);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(static_cast<char*>(G.sel) + 64);
  select_hist_rows(G.A, G.n, shift, bits, st, hist, t.y, t.z, 1);
}

__global__ void k_g_select_step(const GGraph* __restrict__ gs, int shift, int bits, int last) {
  const GGraph& G = gs[blockIdx.x];
  SelectState* st = static_cast<SelectState*>(G.sel);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(static_cast<char*>(G.sel) + 64);
  select_step(st, hist, shift, bits, G.sigma, last);
}

__global__ void k_g_set_sigma(const GGraph* __restrict__ gs, double sigma) { *gs[blockIdx.x].sigma = sigma; }

// tiles: (i << 12) | g, one row per block
__global__ void __launch_bounds__(256) k_g_kernel_rows(const uint32_t* __restrict__ tiles,
                                                        const GGraph* __restrict__ gs) {
  const uint32_t t = tiles[blockIdx.x];
  const GGraph& G = gs[t & 0xFFFu];
  __shared__ double rcp_s;                               // one float64 division per block
  __shared__ ff tab[FF_EXP_TABLE];
  ff_exp_table(tab);
  if (threadIdx.x == 0) {
    const double s = *G.sigma;
    rcp_s = 1.0 / (2.0 * (s * s));
  }
  __syncthreads();
  kernel_row<KERNEL_GAUSSIAN>(G.A, G.n, rcp_s, G.D, (int)(t >> 12), tab);
}

__global__ void k_g_sum(const GGraph* __restrict__ gs) {
  const GGraph& G = gs[blockIdx.x];
  block_sum_to(G.D, G.n, G.vol);
}

}  // namespace

size_t graph_select_bytes() { return 64 + RADIX_BINS * sizeof(unsigned long long); }

void graph_grouped_tiles(const std::vector<int>& n, int T, GraphTiles& out) {
  std::vector<int> order(n.size());
  for (size_t g = 0; g < n.size(); ++g) order[g] = (int)g;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  for (int g : order) {
    const int nn = n[g], nb = (nn + DT - 1) / DT;
    const size_t total = (size_t)nn * T;
    for (size_t b = 0; b * 1024 < total; ++b) out.fixed.push_back(((uint32_t)b << 12) | (uint32_t)g);
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj) out.dist.push_back((uint32_t)g | ((uint32_t)bi << 12) | ((uint32_t)bj << 22));
    // selection: consecutive rows holding about 2^17 upper-triangle keys
    int r0 = 0;
    long long acc = 0;
    for (int i = 0; i < nn - 1; ++i) {
      acc += nn - 1 - i;
      if (acc >= (1 << 17) || i == nn - 2) {
        out.sel.push_back(make_int4(g, r0, i + 1, 0));
        r0 = i + 1;
        acc = 0;
      }
    }
    for (int i = 0; i < nn; ++i) out.rows.push_back(((uint32_t)i << 12) | (uint32_t)g);
  }
}

int graph_build_grouped(cdl_ctx* ctx, const GraphBatch& B) {
  cudaStream_t s = ctx->stream;
  CDL_CUDA_TRY(cudaMemsetAsync(B.sel_all, 0, B.sel_bytes, s));
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_g_select_init<<<B.G2, 1, 0, s>>>(B.gs);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_DISTANCE, 0);
    k_g_to_fixed<<<B.fixed.count, 256, 0, s>>>(B.fixed.p, B.gs);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_DISTANCE, B.dist_terms);
    k_g_dist<<<B.dist.count, 256, 0, s>>>(B.dist.p, B.gs);
    CDL_TRY(L.done());
  }
  if (B.sigma > 0) {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_g_set_sigma<<<B.G2, 1, 0, s>>>(B.gs, B.sigma);
    CDL_TRY(L.done());
  } else {
    const int shifts[6] = {52, 40, 28, 16, 4, 0};
    const int widths[6] = {12, 12, 12, 12, 12, 4};
    for (int p = 0; p < 6; ++p) {
      {
        Launch L(ctx, CDL_KC_SELECT, B.select_bytes);
        k_g_select_hist<<<B.sel_count, 512, 0, s>>>(B.sel, B.gs, shifts[p], widths[p]);
        CDL_TRY(L.done());
      }
      {
        Launch L(ctx, CDL_KC_SELECT, 0);
        k_g_select_step<<<B.G2, 256, 0, s>>>(B.gs, shifts[p], widths[p], p == 5);
        CDL_TRY(L.done());
      }
    }
  }
  {
    Launch L(ctx, CDL_KC_KERNEL, B.kernel_bytes);
    k_g_kernel_rows<<<B.rows.count, 256, 0, s>>>(B.rows.p, B.gs);
    CDL_TRY(L.done());
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_g_sum<<<B.G2, 1024, 0, s>>>(B.gs);
  return L.done();
}

int graph_build(cdl_ctx* ctx, const double* X, int64_t n64, int T, double sigma, double* A,
                double* D, double* vol, double* sigma_out, int kernel, unsigned long long* amax_bits) {
  const int n = (int)n64;
  cudaStream_t s = ctx->stream;
  void *wsXi, *wsSt, *wsHist;
  CDL_TRY(ws_get(ctx, "graph.Xi", (size_t)n * T * sizeof(int), &wsXi));
  CDL_TRY(ws_get(ctx, "graph.state", sizeof(SelectState), &wsSt));
  CDL_TRY(ws_get(ctx, "graph.hist", RADIX_BINS * sizeof(unsigned long long), &wsHist));
  SelectState* st = static_cast<SelectState*>(wsSt);
  unsigned long long* hist = static_cast<unsigned long long*>(wsHist);
  const long long m = (long long)n * (n - 1) / 2;
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_select_init<<<1, 1, 0, s>>>(st, (m - 1) / 2);
    CDL_TRY(L.done());
  }
  CDL_CUDA_TRY(cudaMemsetAsync(hist, 0, RADIX_BINS * sizeof(unsigned long long), s));
  {
    size_t total = (size_t)n * T;
    int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->sm_count * 8);
    Launch L(ctx, CDL_KC_DISTANCE, 0);
    k_to_fixed<<<blocks, 256, 0, s>>>(X, static_cast<int*>(wsXi), n, T, st);
    CDL_TRY(L.done());
  }
  const int nb = (n + DT - 1) / DT;
  const long long tiles = (long long)nb * (nb + 1) / 2;
  if (tiles > 0x7fffffffLL) return CDL_ERR_INVALID_ARG;
  {
    // grid inputs: exact Gram on the tensor cores (three bf16 digit planes)
    const int rows = (n + 127) / 128 * 128, tp = (T + 63) / 64 * 64;
    void *wsPl, *wsNo;
    CDL_TRY(ws_get(ctx, "graph.xplanes", 3 * (size_t)rows * tp * 2, &wsPl));
    CDL_TRY(ws_get(ctx, "graph.norms", (size_t)rows * sizeof(long long), &wsNo));
    {
      Launch L(ctx, CDL_KC_DISTANCE, 0);
      const size_t cnt = (size_t)rows * tp;
      k_slice_x<<<(unsigned)std::min<size_t>((cnt + 255) / 256, (size_t)ctx->sm_count * 8), 256, 0, s>>>(
          X, n, T, rows, tp, static_cast<__nv_bfloat16*>(wsPl));
      CDL_TRY(L.done());
    }
    {
      Launch L(ctx, CDL_KC_DISTANCE, 0);
      k_row_norms<<<rows / 8, 256, 0, s>>>(X, n, T, rows, static_cast<long long*>(wsNo));
      CDL_TRY(L.done());
    }
    CDL_TRY(dist_tc(ctx, wsPl, static_cast<const long long*>(wsNo), n, rows, tp, A, &st->flags,
                    0.5 * (double)n * (double)(n - 1) * T));
  }
  {
    Launch L(ctx, CDL_KC_DISTANCE, 0);
    k_dist_f64<<<(unsigned)tiles, 256, 0, s>>>(X, n, T, A, st);
    CDL_TRY(L.done());
  }
  if (sigma > 0) {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_set_scalar<<<1, 1, 0, s>>>(sigma_out, sigma);
    CDL_TRY(L.done());
  } else {
    // digits from the top: [52,64), [40,52), [28,40), [16,28), [4,16), [0,4)
    const int shifts[6] = {52, 40, 28, 16, 4, 0};
    const int widths[6] = {12, 12, 12, 12, 12, 4};
    const int hblocks = std::min(n - 1, ctx->sm_count * 4);
    const long long cap = std::min(SELECT_CAP, std::max(m / 64, 1024ll));
    void* wsBuf;
    CDL_TRY(ws_get(ctx, "graph.selbuf", (size_t)cap * sizeof(unsigned long long), &wsBuf));
    unsigned long long* sbuf = static_cast<unsigned long long*>(wsBuf);
    for (int p = 0; p < 6; ++p) {
      {
        // work: bytes of the triangle for the full passes (the later ones read the copied keys)
        Launch L(ctx, CDL_KC_SELECT, p < 3 ? 8.0 * (double)m : 0.0);
        if (p < 2)
          k_select_hist<<<hblocks, 512, 0, s>>>(A, n, shifts[p], widths[p], st, hist);
        else if (p == 2)
          k_select_hist_compact<<<hblocks, 512, 0, s>>>(A, n, shifts[p], widths[p], st, hist, sbuf, cap);
        else
          k_select_hist_buf<<<hblocks, 512, 0, s>>>(A, n, shifts[p], widths[p], st, hist, sbuf, cap);
        CDL_TRY(L.done());
      }
      {
        Launch L(ctx, CDL_KC_SELECT, 0);
        k_select_step<<<1, 256, 0, s>>>(st, hist, shifts[p], widths[p], sigma_out, p == 5);
        CDL_TRY(L.done());
      }
    }
  }
  {
    void* wsPart;
    CDL_TRY(ws_get(ctx, "graph.dpart", (size_t)nb * n * sizeof(double), &wsPart));
    double* part = static_cast<double*>(wsPart);
    if (amax_bits) CDL_CUDA_TRY(cudaMemsetAsync(amax_bits, 0, sizeof(unsigned long long), s));
    {
      Launch L(ctx, CDL_KC_KERNEL, 16.0 * (double)n * n);
      if (kernel == KERNEL_EXP)
        k_kernel_tiles<KERNEL_EXP><<<(unsigned)tiles, 256, 0, s>>>(A, n, sigma_out, part, amax_bits);
      else
        k_kernel_tiles<KERNEL_GAUSSIAN><<<(unsigned)tiles, 256, 0, s>>>(A, n, sigma_out, part, amax_bits);
      CDL_TRY(L.done());
    }
    Launch L(ctx, CDL_KC_MISC, 0);
    k_part_sums<<<(n + 255) / 256, 256, 0, s>>>(part, nb, n, D);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_sum<<<1, 1024, 0, s>>>(D, n, vol);
    CDL_TRY(L.done());
  }
  return CDL_OK;
}

// ---------------------------------------------------------------------------
// Graphs too large to keep: the Gaussian-kernel graph regenerated from the
// node series in row panels of P rows wherever it is needed. The series'
// digit planes and squared norms are formed once (distances exact on the
// tensor cores; inputs must lie on the 2^-16 grid), sigma by the same exact
// radix select as graph_build with every histogram pass streaming the
// upper-triangle part of each panel's distances, then the degrees from the
// panels' kernel rows. The panel A values equal graph_build's (exact
// distances, the same exponential), the degrees up to summation order.
int graph_regen_init(cdl_ctx* ctx, RegenGraph& g, const double* X, int64_t n64, int T, double sigma, double* panel,
                     int P) {
  const int n = (int)n64;
  cudaStream_t s = ctx->stream;
  g.X = X;
  g.n = n;
  g.T = T;
  g.rows = (n + 127) / 128 * 128;
  g.tp = (T + 63) / 64 * 64;
  const std::string tag = "regen." + std::to_string(g.id) + ".";
  void *wsXi, *wsSt, *wsHist, *wsPl, *wsNo, *wsSc;
  CDL_TRY(ws_get(ctx, (tag + "Xi").c_str(), (size_t)n * T * sizeof(int), &wsXi));
  CDL_TRY(ws_get(ctx, (tag + "state").c_str(), sizeof(SelectState), &wsSt));
  CDL_TRY(ws_get(ctx, (tag + "hist").c_str(), RADIX_BINS * sizeof(unsigned long long), &wsHist));
  CDL_TRY(ws_get(ctx, (tag + "planes").c_str(), 3 * (size_t)g.rows * g.tp * 2, &wsPl));
  CDL_TRY(ws_get(ctx, (tag + "norms").c_str(), (size_t)g.rows * sizeof(long long), &wsNo));
  CDL_TRY(ws_get(ctx, (tag + "scalars").c_str(), 2 * sizeof(double), &wsSc));
  SelectState* st = static_cast<SelectState*>(wsSt);
  unsigned long long* hist = static_cast<unsigned long long*>(wsHist);
  g.planes = wsPl;
  g.norms = static_cast<const long long*>(wsNo);
  g.offgrid = &st->flags;
  g.sigma = static_cast<double*>(wsSc);
  const long long m = (long long)n * (n - 1) / 2;
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_select_init<<<1, 1, 0, s>>>(st, (m - 1) / 2);
    CDL_TRY(L.done());
  }
  CDL_CUDA_TRY(cudaMemsetAsync(hist, 0, RADIX_BINS * sizeof(unsigned long long), s));
  {
    const size_t total = (size_t)n * T;
    Launch L(ctx, CDL_KC_DISTANCE, 0);
    k_to_fixed<<<(int)std::min<size_t>((total + 255) / 256, (size_t)ctx->sm_count * 8), 256, 0, s>>>(
        X, static_cast<int*>(wsXi), n, T, st);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_DISTANCE, 0);
    const size_t cnt = (size_t)g.rows * g.tp;
    k_slice_x<<<(unsigned)std::min<size_t>((cnt + 255) / 256, (size_t)ctx->sm_count * 8), 256, 0, s>>>(
        X, n, T, g.rows, g.tp, static_cast<__nv_bfloat16*>(wsPl));
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_DISTANCE, 0);
    k_row_norms<<<g.rows / 8, 256, 0, s>>>(X, n, T, g.rows, static_cast<long long*>(wsNo));
    CDL_TRY(L.done());
  }
  int flags = 0;
  CDL_CUDA_TRY(cudaMemcpyAsync(&flags, &st->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CDL_CUDA_TRY(cudaStreamSynchronize(s));
  if (flags & 1) {
    set_last_error("graph regeneration needs inputs on the 2^-16 grid", __FILE__, __LINE__);
    return CDL_ERR_UNSUPPORTED;
  }
  if (sigma > 0) {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_set_scalar<<<1, 1, 0, s>>>(g.sigma, sigma);
    CDL_TRY(L.done());
  } else {
    const int shifts[6] = {52, 40, 28, 16, 4, 0};
    const int widths[6] = {12, 12, 12, 12, 12, 4};
    for (int p = 0; p < 6; ++p) {
      for (int r0 = 0; r0 < g.rows; r0 += P) {
        const int pr = std::min(P, g.rows - r0);
        CDL_TRY(dist_tc_panel(ctx, g.planes, g.norms, n, g.rows, g.tp, panel, r0, pr, true, g.offgrid));
        const int r1 = std::min(n - 1, r0 + pr);
        if (r1 <= r0) continue;
        Launch L(ctx, CDL_KC_SELECT, 8.0 * (double)pr * n);
        k_select_hist_panel<<<std::min(r1 - r0, ctx->sm_count * 4), 512, 0, s>>>(panel, n, shifts[p], widths[p], st,
                                                                               hist, r0, r1);
        CDL_TRY(L.done());
      }
      Launch L(ctx, CDL_KC_SELECT, 0);
      k_select_step<<<1, 256, 0, s>>>(st, hist, shifts[p], widths[p], g.sigma, p == 5);
      CDL_TRY(L.done());
    }
  }
  // degrees: every panel's kernel rows once
  for (int r0 = 0; r0 < n; r0 += P) {
    const int pr = std::min(P, n - r0);
    CDL_TRY(regen_panel(ctx, g, panel, r0, pr, g.D));
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_sum<<<1, 1024, 0, s>>>(g.D, n, g.vol);
  return L.done();
}

int regen_panel(cdl_ctx* ctx, const RegenGraph& g, double* panel, int r0, int rows, double* D) {
  const int pr = (int)std::min<long long>(round_up(rows, 128), g.rows - r0);
  CDL_TRY(dist_tc_panel(ctx, g.planes, g.norms, g.n, g.rows, g.tp, panel, r0, pr, false, g.offgrid));
  const int r1 = std::min(g.n, r0 + rows);
  Launch L(ctx, CDL_KC_KERNEL, 16.0 * (double)(r1 - r0) * g.n);
  k_kernel_rows_panel<<<std::min(r1 - r0, ctx->sm_count * 8), 256, 0, ctx->stream>>>(panel, g.n, g.sigma, D, r0, r1);
  return L.done();
}

// ---------------------------------------------------------------------------
// Given graphs: degrees of a caller's adjacency matrix and symmetric edge
// weights added to it (the second graph of the synthetic experiments,
// A_2 = Q + (R + R^T) / 2, Sec. 4.2.1).

// D_i = sum_j A_ij, one block (256 threads) per row: each thread adds its
// strided terms in float64 with a running compensation (Neumaier's TwoSum
// form), the (sum, compensation) pairs are combined the same way across the
// warp and the block; D_i = sum + compensation (within a few units in the
// last place of the exact row sum).
__device__ __forceinline__ void neumaier_add(double& s, double& c, double a) {
  const double t = s + a;
  c += fabs(s) >= fabs(a) ? (s - t) + a : (a - t) + s;
  s = t;
}

__global__ void __launch_bounds__(256) k_degrees(const double* __restrict__ A, int n, double* __restrict__ D) {
  __shared__ double red_s[8], red_c[8];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const double* row = A + (size_t)i * n;
    double s = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < n; j += 256) neumaier_add(s, c, row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
      neumaier_add(s, c, s2);
      c += c2;
    }
    if ((threadIdx.x & 31) == 0) {
      red_s[threadIdx.x >> 5] = s;
      red_c[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = red_s[0], tc = red_c[0];
      for (int w = 1; w < 8; ++w) {
        neumaier_add(t, tc, red_s[w]);
        tc += red_c[w];
      }
      D[i] = t + tc;
    }
    __syncthreads();
  }
}

// A_ij += w_e and A_ji += w_e for each pair e = (i, j) of ij (m x 2, row-major).
// Invalid entries (an index outside [0, n), i == j, w negative, infinite or
// NaN) are skipped and counted in *bad. Each listed unordered pair touches its
// two entries once, so distinct pairs give exact, order-free results.
__global__ void k_add_edges(double* __restrict__ A, int n, long long m, const long long* __restrict__ ij,
                            const double* __restrict__ w, unsigned long long* __restrict__ bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const long long i = ij[2 * e], j = ij[2 * e + 1];
    const double v = w[e];
    if (i < 0 || i >= n || j < 0 || j >= n || i == j || !(v >= 0.0) || isinf(v)) {
      atomicAdd(bad, 1ull);
      continue;
    }
    atomicAdd(A + (size_t)i * n + j, v);
    atomicAdd(A + (size_t)j * n + i, v);
  }
}

int graph_degrees(cdl_ctx* ctx, const double* A, int64_t n64, double* D, double* vol) {
  const int n = (int)n64;
  cudaStream_t s = ctx->stream;
  {
    Launch L(ctx, CDL_KC_KERNEL, 8.0 * (double)n * n);
    k_degrees<<<std::min(n, ctx->sm_count * 8), 256, 0, s>>>(A, n, D);
    CDL_TRY(L.done());
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_sum<<<1, 1024, 0, s>>>(D, n, vol);
  return L.done();
}

int graph_add_edges(cdl_ctx* ctx, double* A, int64_t n, int64_t m, const int64_t* ij, const double* w,
                    int64_t* n_bad) {
  cudaStream_t s = ctx->stream;
  void* wsBad;
  CDL_TRY(ws_get(ctx, "graph.bad", sizeof(unsigned long long), &wsBad));
  unsigned long long* bad = static_cast<unsigned long long*>(wsBad);
  CDL_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
  if (m > 0) {
    const long long blocks = std::min<long long>((m + 255) / 256, (long long)ctx->sm_count * 16);
    Launch L(ctx, CDL_KC_MISC, 0);
    k_add_edges<<<(unsigned)blocks, 256, 0, s>>>(A, (int)n, (long long)m, reinterpret_cast<const long long*>(ij),
                                                 w, bad);
    CDL_TRY(L.done());
  }
  unsigned long long h = 0;
  CDL_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
  CDL_CUDA_TRY(cudaStreamSynchronize(s));
  if (n_bad) *n_bad = (int64_t)h;
  return h ? CDL_ERR_INVALID_ARG : CDL_OK;
}

// ---------------------------------------------------------------------------
// Graph build without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a process that has
// handed (almost) all device memory to its own pool allocator, where an extra
// allocation would fail or fragment the pool, or a service that must not
// allocate once it is running. For them cdl_build_graph_static runs the same
// kernels as cdl_build_graph, with all of their scratch (the fixed-point copy
// of X, the radix-select state and histogram) in the statically allocated
// device array below, which every GPU that loads the library holds until the
// process exits. The caller still owns X and the outputs.

constexpr size_t STATIC_XT_ELEMS = size_t(1) << 20;   // n * T limit (4 MiB of int32)
constexpr size_t STATIC_HIST_OFF = STATIC_XT_ELEMS * sizeof(int);
constexpr size_t STATIC_STATE_OFF = STATIC_HIST_OFF + RADIX_BINS * sizeof(unsigned long long);
constexpr size_t STATIC_SCRATCH_BYTES = STATIC_STATE_OFF + 256;

static __device__ __align__(256) unsigned char g_graph_scratch[STATIC_SCRATCH_BYTES];

namespace {

// The device address of g_graph_scratch belongs to the CUDA context that was
// current when it was looked up: another context on the same device (one the
// caller made current through the driver API, or the primary context
// re-created after cudaDeviceReset) has its own copy of the array at another
// address. So the address is cached per context, keyed by the context's
// unique ID (cuCtxGetId: IDs are never reused within a process), and the
// host-side name of the array, which is only a stand-in for the symbol, is
// never passed to a kernel.
constexpr int MAX_CONTEXTS = 64;
std::mutex g_static_mu;
unsigned long long g_static_ctx_id[MAX_CONTEXTS] = {0};
void* g_static_addr[MAX_CONTEXTS] = {nullptr};
int g_static_used = 0;

typedef int (*PFN_ctx_get_current)(void** ctx);
typedef int (*PFN_ctx_get_id)(void* ctx, unsigned long long* id);

// ID of the current CUDA context. Driver entry points are taken through the
// runtime, so the library does not link libcuda itself.
int current_context_id(unsigned long long* id) {
  static PFN_ctx_get_current get_current = nullptr;
  static PFN_ctx_get_id get_id = nullptr;
  if (!get_current || !get_id) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return CDL_ERR_CUDA;
    get_current = reinterpret_cast<PFN_ctx_get_current>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return CDL_ERR_CUDA;
    get_id = reinterpret_cast<PFN_ctx_get_id>(p);
  }
  // the pointer checks before this call have already made the runtime's
  // context current when the caller had none
  void* c = nullptr;
  if (get_current(&c) != 0 || !c) {
    set_last_error("no current CUDA context", __FILE__, __LINE__);
    return CDL_ERR_CUDA;
  }
  if (get_id(c, id) != 0) {
    set_last_error("cuCtxGetId failed", __FILE__, __LINE__);
    return CDL_ERR_CUDA;
  }
  return CDL_OK;
}

// Device address of g_graph_scratch in the current context, looked up with
// that context current on the first call in it and cached.
int static_scratch(void** out) {
  unsigned long long id = 0;
  CDL_TRY(current_context_id(&id));
  std::lock_guard<std::mutex> lock(g_static_mu);
  for (int i = 0; i < g_static_used; ++i)
    if (g_static_ctx_id[i] == id) {
      *out = g_static_addr[i];
      return CDL_OK;
    }
  void* p = nullptr;
  CDL_CUDA_TRY(cudaGetSymbolAddress(&p, g_graph_scratch));
  // a full table starts over: the contexts it names may be gone, and a
  // lookup costs one symbol query
  if (g_static_used == MAX_CONTEXTS) g_static_used = 0;
  g_static_ctx_id[g_static_used] = id;
  g_static_addr[g_static_used] = p;
  ++g_static_used;
  *out = p;
  return CDL_OK;
}

// Device or managed memory reachable from the current device (the same
// rule as the context-based entry points).
int on_current_device(const void* p) {
  if (!p) return CDL_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(p) % 8) return CDL_ERR_INVALID_ARG;
  int dev = 0;
  CDL_CUDA_TRY(cudaGetDevice(&dev));
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return CDL_ERR_INVALID_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return CDL_ERR_INVALID_ARG;
  if (at.type == cudaMemoryTypeDevice && at.device != dev) return CDL_ERR_INVALID_ARG;
  return CDL_OK;
}

int launched() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return CDL_ERR_CUDA;
  }
  return CDL_OK;
}

}  // namespace

int graph_build_static(const double* X, int64_t n64, int T, double sigma, double* A, double* D,
                       double* vol, double* sigma_out, cudaStream_t s) {
  if (n64 < 2 || n64 > (1 << 20) || T < 1 || T > 4096) return CDL_ERR_INVALID_ARG;
  if ((size_t)n64 * (size_t)T > STATIC_XT_ELEMS) {
    set_last_error("n * T exceeds the static scratch limit of 2^20 samples", __FILE__, __LINE__);
    return CDL_ERR_INVALID_ARG;
  }
  CDL_TRY(on_current_device(X));
  CDL_TRY(on_current_device(A));
  CDL_TRY(on_current_device(D));
  CDL_TRY(on_current_device(vol));
  CDL_TRY(on_current_device(sigma_out));
  void* base = nullptr;
  CDL_TRY(static_scratch(&base));
  int dev = 0, sm_count = 0;
  CDL_CUDA_TRY(cudaGetDevice(&dev));
  CDL_CUDA_TRY(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
  const int n = (int)n64;
  int* Xt = static_cast<int*>(base);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(static_cast<char*>(base) + STATIC_HIST_OFF);
  SelectState* st = reinterpret_cast<SelectState*>(static_cast<char*>(base) + STATIC_STATE_OFF);
  const long long m = (long long)n * (n - 1) / 2;
  // The array keeps the previous call's contents: the select state and the
  // histogram must start from zero, Xt is fully overwritten.
  k_select_init<<<1, 1, 0, s>>>(st, (m - 1) / 2);
  CDL_TRY(launched());
  CDL_CUDA_TRY(cudaMemsetAsync(hist, 0, RADIX_BINS * sizeof(unsigned long long), s));
  const size_t total = (size_t)n * T;
  k_to_fixed<<<(int)std::min<size_t>((total + 255) / 256, (size_t)sm_count * 8), 256, 0, s>>>(X, Xt, n, T, st);
  CDL_TRY(launched());
  const int nb = (n + DT - 1) / DT;
  const long long tiles = (long long)nb * (nb + 1) / 2;
  k_dist_int<<<(unsigned)tiles, 256, 0, s>>>(Xt, n, T, A, st);
  CDL_TRY(launched());
  k_dist_f64<<<(unsigned)tiles, 256, 0, s>>>(X, n, T, A, st);
  CDL_TRY(launched());
  if (sigma > 0) {
    k_set_scalar<<<1, 1, 0, s>>>(sigma_out, sigma);
    CDL_TRY(launched());
  } else {
    const int shifts[6] = {52, 40, 28, 16, 4, 0};
    const int widths[6] = {12, 12, 12, 12, 12, 4};
    const int hblocks = std::min(n - 1, sm_count * 4);
    for (int p = 0; p < 6; ++p) {
      k_select_hist<<<hblocks, 512, 0, s>>>(A, n, shifts[p], widths[p], st, hist);
      CDL_TRY(launched());
      k_select_step<<<1, 256, 0, s>>>(st, hist, shifts[p], widths[p], sigma_out, p == 5);
      CDL_TRY(launched());
    }
  }
  k_kernel_rows<KERNEL_GAUSSIAN><<<std::min(n, sm_count * 8), 256, 0, s>>>(A, n, sigma_out, D);
  CDL_TRY(launched());
  k_sum<<<1, 1024, 0, s>>>(D, n, vol);
  return launched();
}

}  // namespace cdl
