// Random projection Y = (Q W^{1/2} B)^T of Alg. 1 ("y = W^{1/2} B q") and
// Alg. 3, formed edge by edge without materialising B or Q (the Map +
// ReduceByKey of Sec. 4.1):
//   Y[i, r] = k^{-1/2} sum_{j != i} o_ij s_r(min(i,j), max(i,j)) sqrt(A_ij),
// o_ij = +1 when i < j (i is the head of edge (i, j), Sec. 2), else -1.
// The signs come from Philox4x32-10 (Salmon et al., SC'11) at counter
// (i, j, r / 128, 0) with key (seed low word, seed high word): bit (r mod 32)
// of output word ((r mod 128) / 32) set means +1.
//
// Each thread owns one node row i and 16 projection rows (half a Philox word).
// Per tile of 32 edges the block forms sqrt(A_ij) in float-float once per
// (row, edge) and one Philox call per (row, edge, 128 projection rows), shared
// through shared memory by the threads of the row.
#include <algorithm>
#include <cmath>

#include "ff.cuh"
#include "internal.h"

namespace cdl {
namespace {

constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;   // golden-ratio Weyl increment
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;   // sqrt(3) - 1 Weyl increment

// Philox4x32 with 10 rounds: per round, words 0 and 2 are multiplied by the
// two constants; the high halves are mixed with words 1, 3 and the round key,
// the low halves become words 1 and 3; the key advances between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    const uint32_t lo0 = PHILOX_M0 * c.x, hi0 = __umulhi(PHILOX_M0, c.x);
    const uint32_t lo1 = PHILOX_M1 * c.z, hi1 = __umulhi(PHILOX_M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

constexpr int JT = 32;       // j-tile
constexpr int JTP = JT + 1;  // padded row stride of the piece arrays: the node rows of a warp fall in different banks
constexpr int CHUNK = 4096;  // exact float32 accumulation length (multiple of JT)
constexpr int MAX_RPB = 64;  // node rows per block

// Each (node row i, edge j) term o_ij sqrt(A_ij) is split into three float
// pieces p1 + p2 + p3: with 2^h (h >= 0) the least power of two not below
// sqrt(max A) (h = 0 for kernel graphs, whose weights are at most 1), p1 on
// the 2^(h-12) grid (|p1| <= 2^h), p2 on the 2^(h-24) grid (|p2| <= 2^(h-13))
// and the remainder p3 (|p3| <= 2^(h-24)). Signed sums of up to 4096 p1 (or
// p2) values stay on their grid below 2^24 grid steps, so float32 adds them
// exactly; p3 is small enough for plain float32 sums. The three partial sums
// are flushed to float64 in Y every 4096 edges. Per term and projection row
// this is one bit test and three predicated adds (the terms with a set sign
// bit; the plain totals are kept once per row and combined at the flush).
constexpr int RB = 16;       // projection rows per thread (half a Philox word)

// Shared memory of a block: three piece arrays [rpb][JTP] floats, then (16-byte
// aligned) the Philox words [rpb][JT * nrb + 1] (the extra word staggers banks).
__host__ __device__ inline size_t project_words_offset(int rpb) {
  return ((size_t)3 * rpb * JTP * sizeof(float) + 15) / 16 * 16;
}
__host__ __device__ inline size_t project_smem_bytes(int rpb, int W) {
  const int nrb = (W + 3) / 4;
  return project_words_offset(rpb) + (size_t)rpb * (JT * nrb + 1) * sizeof(uint4);
}

// Rows [bidx * rpb, bidx * rpb + rpb) of Y over the edges to nodes j in
// [jbeg, jend) (jbeg a multiple of CHUNK): written, not accumulated, and
// multiplied by `scale` when `final` (otherwise left unscaled: a partial sum).
// With a row window [r0, r1) (r1 > 0) the rows are r0 + bidx * rpb ... < r1
// and A holds rows r0 .. (A[(i - r0) n + j]).
__device__ __forceinline__ void project_rows_block(const double* __restrict__ A, int n, int k, int W, int rpb,
                                                   uint32_t key0, uint32_t key1, double scale,
                                                   double* __restrict__ Y, int bidx, int gexp, int jbeg, int jend,
                                                   bool final, int r0 = 0, int r1 = 0) {
  // piece grids 2^(gexp - 12) and 2^(gexp - 24) (gexp = h of the comment above)
  const float up1 = __int_as_float((127 + 12 - gexp) << 23), dn1 = __int_as_float((127 - 12 + gexp) << 23);
  const float up2 = __int_as_float((127 + 24 - gexp) << 23), dn2 = __int_as_float((127 - 24 + gexp) << 23);
  extern __shared__ __align__(16) unsigned char smraw[];
  float* P1 = reinterpret_cast<float*>(smraw);          // [rpb][JTP]
  float* P2 = P1 + rpb * JTP;                           // [rpb][JTP]
  float* P3 = P2 + rpb * JTP;                           // [rpb][JTP]
  uint4* Wd = reinterpret_cast<uint4*>(smraw + project_words_offset(rpb));   // [rpb][WS]
  const int nrb = (W + 3) / 4;
  const int WS = JT * nrb + 1;
  const int H = 2 * W;                 // threads per node row
  const int t = threadIdx.x;
  const int rl = t / H, h = t % H;
  const int w = h >> 1, shift = (h & 1) * RB;
  const int rend = r1 > 0 ? r1 : n;
  const int i0 = r0 + bidx * rpb;
  const int i = i0 + rl;
  const bool active = rl < rpb && i < rend;
  // With s = 2 bit - 1, sum_j s x_j = 2 sum_{bit set} x_j - sum_j x_j: the
  // a-accumulators take the terms whose sign bit is set (one predicated add per
  // piece), t the plain totals (shared by all projection rows of the thread).
  float a1[RB], a2[RB], a3[RB];
  float t1 = 0.f, t2 = 0.f, t3 = 0.f;
#pragma unroll
  for (int b = 0; b < RB; ++b) a1[b] = a2[b] = a3[b] = 0.f;
  bool first = true;
  auto flush = [&]() {
    if (!active) return;
    const double s1 = t1, s2 = t2, s3 = t3;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const int r = w * 32 + shift + b;
      // exact in float64 for the two grid pieces
      const double v = ((2.0 * (double)a1[b] - s1) + (2.0 * (double)a2[b] - s2)) + (2.0 * (double)a3[b] - s3);
      if (r < k) Y[(size_t)i * k + r] = first ? v : Y[(size_t)i * k + r] + v;
      a1[b] = a2[b] = a3[b] = 0.f;
    }
    t1 = t2 = t3 = 0.f;
    first = false;
  };
  for (int j0 = jbeg; j0 < jend; j0 += JT) {
    if (j0 > jbeg && j0 % CHUNK == 0) flush();
    __syncthreads();
    // pieces of o_ij sqrt(A_ij) for the tile
    for (int e = t; e < rpb * JT; e += blockDim.x) {
      const int rr = e / JT, jj = e % JT;
      const int ii = i0 + rr, j = j0 + jj;
      float p1 = 0.f, p2 = 0.f, p3 = 0.f;
      if (ii < rend && j < jend && j != ii) {
        const ff a = split_nonneg(A[(size_t)(ii - r0) * n + j]);   // integer split, no float64 ops
        const float ah = a.hi, al = a.lo;
        if (ah > 0.f) {
          // sqrt(ah + al) = sh + sl with sl = (ah - sh^2 + al) / (2 sh)
          const float sh = __fsqrt_rn(ah);
          const float res = __fadd_rn(__fmaf_rn(-sh, sh, ah), al);
          const float sl = __fmul_rn(res, __fdiv_rn(0.5f, sh));
          p1 = __fmul_rn(rintf(__fmul_rn(sh, up1)), dn1);
          const float rem = __fsub_rn(sh, p1);                   // exact
          p2 = __fmul_rn(rintf(__fmul_rn(rem, up2)), dn2);
          p3 = __fadd_rn(__fsub_rn(rem, p2), sl);
          if (j < ii) {   // ii is the tail of edge (j, ii)
            p1 = -p1;
            p2 = -p2;
            p3 = -p3;
          }
        }
      }
      P1[rr * JTP + jj] = p1;
      P2[rr * JTP + jj] = p2;
      P3[rr * JTP + jj] = p3;
    }
    // Philox words: one call per (row, edge, 128-row block of the projection)
    for (int c = t; c < rpb * JT * nrb; c += blockDim.x) {
      const int rb = c % nrb, e = c / nrb;
      const int rr = e / JT, jj = e % JT;
      const int ii = i0 + rr, j = j0 + jj;
      uint4 o = make_uint4(0u, 0u, 0u, 0u);
      if (ii < rend && j < jend && j != ii)
        o = philox4x32_10(make_uint4((uint32_t)min(ii, j), (uint32_t)max(ii, j), (uint32_t)rb, 0u), key0, key1);
      Wd[rr * WS + jj * nrb + rb] = o;
    }
    __syncthreads();
    if (!active) continue;
    const int jmax = min(JT, jend - j0);
    const int wi = w & 3, rb = w >> 2;
    const uint32_t* Ww = reinterpret_cast<const uint32_t*>(Wd + rl * WS + rb) + wi;   // this thread's word
#pragma unroll 2
    for (int jj = 0; jj < jmax; ++jj) {
      const int e = rl * JTP + jj;
      const float p1 = P1[e], p2 = P2[e], p3 = P3[e];
      const uint32_t bits = Ww[jj * nrb * 4] >> shift;   // set bit -> +1
      t1 = __fadd_rn(t1, p1);
      t2 = __fadd_rn(t2, p2);
      t3 = __fadd_rn(t3, p3);
#pragma unroll
      for (int b = 0; b < RB; ++b)
        asm("{\n\t.reg .pred q;\n\t"
            "setp.ne.b32 q, %3, 0;\n\t"
            "@q add.rn.f32 %0, %0, %4;\n\t"
            "@q add.rn.f32 %1, %1, %5;\n\t"
            "@q add.rn.f32 %2, %2, %6;\n\t}"
            : "+f"(a1[b]), "+f"(a2[b]), "+f"(a3[b])
            : "r"(bits & (1u << b)), "f"(p1), "f"(p2), "f"(p3));
    }
  }
  flush();
  if (!active || !final) return;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    const int r = w * 32 + shift + b;
    if (r < k) Y[(size_t)i * k + r] *= scale;
  }
}

// Grid (row blocks, splits): split s covers the edge chunk [s CHUNK, (s + 1)
// CHUNK) and, with more than one split, writes its unscaled partial sums to
// Y + s n k (k_project_sum adds them in split order, which is the order in
// which one block would have flushed its chunks, and scales).
__global__ void __launch_bounds__(256, 2) k_project(const double* __restrict__ A, int n, int k, int W, int rpb,
                                                     uint32_t key0, uint32_t key1, double scale,
                                                     double* __restrict__ Y,
                                                     const unsigned long long* __restrict__ amax_bits) {
  const int h = min((pow2_exp_above(*amax_bits) + 1) / 2, 100);   // sqrt(max A) <= 2^h (A < 2^200)
  const int split = blockIdx.y, nsplit = gridDim.y;
  const int jbeg = split * CHUNK, jend = nsplit == 1 ? n : min(n, jbeg + CHUNK);
  project_rows_block(A, n, k, W, rpb, key0, key1, scale, Y + (size_t)split * n * k, blockIdx.x, h, jbeg, jend,
                     nsplit == 1);
}

// Rows r0 .. r1 - 1 of Y (unscaled sums, then scaled) from a panel holding
// those rows of A (A[(i - r0) n + j]); block b covers rows r0 + b rpb ...
__global__ void __launch_bounds__(256, 2) k_project_panel(const double* __restrict__ P, int n, int k, int W, int rpb,
                                                           uint32_t key0, uint32_t key1, double scale,
                                                           double* __restrict__ Y,
                                                           const unsigned long long* __restrict__ amax_bits, int r0,
                                                           int r1) {
  const int h = min((pow2_exp_above(*amax_bits) + 1) / 2, 100);
  project_rows_block(P, n, k, W, rpb, key0, key1, scale, Y, blockIdx.x, h, 0, n, true, r0, r1);
}

__global__ void k_project_sum(const double* __restrict__ part, int nsplit, size_t count, double scale,
                              double* __restrict__ Y) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    double v = part[idx];
    for (int s = 1; s < nsplit; ++s) v += part[(size_t)s * count + idx];
    Y[idx] = v * scale;
  }
}

// Column sums of Y over 256-row chunks (fixed order): part[b][r].
__device__ __forceinline__ void colsum_chunk(const double* __restrict__ Y, int n, int k, double* __restrict__ part,
                                             int b) {
  __shared__ double sh[8][33];
  const int i0 = b * 256, i1 = min(n, i0 + 256);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r0 = 0; r0 < k; r0 += 32) {
    const int r = r0 + tx;
    double acc = 0.0;
    if (r < k)
      for (int i = i0 + ty; i < i1; i += 8) acc += Y[(size_t)i * k + r];
    sh[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && r < k) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += sh[q][tx];
      part[(size_t)b * k + r] = t;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_colsum(const double* __restrict__ Y, int n, int k,
                                                 double* __restrict__ part) {
  colsum_chunk(Y, n, k, part, blockIdx.x);
}

// Y -= column mean. The exact Y has zero column sums (each edge adds +x to
// its head's row and -x to its tail's); the float sums of the two rows round
// differently, and that residue lies in the null space of L, where no
// solution Z can match it.
__device__ __forceinline__ void sub_mean(double* __restrict__ Y, int n, int k, const double* __restrict__ part,
                                         int nparts, size_t idx) {
  if (idx >= (size_t)n * k) return;
  const int r = (int)(idx % k);
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += part[(size_t)q * k + r];
  Y[idx] -= s / n;
}

// Column means once per column (the same ordered sums as sub_mean), then the subtraction.
__global__ void k_col_mean(const double* __restrict__ part, int nparts, int n, int k, double* __restrict__ mean) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += part[(size_t)q * k + r];
  mean[r] = s / n;
}

__global__ void k_sub_mean(double* __restrict__ Y, int n, int k, const double* __restrict__ mean) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx < (size_t)n * k) Y[idx] -= mean[idx % k];
}

// ---------------------------------------------------------------- batched form
__global__ void __launch_bounds__(256, 2) k_g_project(const uint32_t* __restrict__ tiles, const PGraph* __restrict__ gs,
                                                       int k, int W, int rpb, uint32_t key0, uint32_t key1,
                                                       double scale) {
  const uint32_t t = tiles[blockIdx.x];
  const PGraph& G = gs[t & 0xFFFu];
  project_rows_block(G.A, G.n, k, W, rpb, key0, key1, scale, G.Y, (int)(t >> 12), 0, 0, G.n,
                     true);   // kernel graphs: A <= 1
}

__global__ void __launch_bounds__(256) k_g_colsum(const uint32_t* __restrict__ tiles, const PGraph* __restrict__ gs,
                                                   int k) {
  const uint32_t t = tiles[blockIdx.x];
  const PGraph& G = gs[t & 0xFFFu];
  colsum_chunk(G.Y, G.n, k, G.part, (int)(t >> 12));
}

__global__ void k_g_sub_mean(const uint32_t* __restrict__ tiles, const PGraph* __restrict__ gs, int k) {
  const uint32_t t = tiles[blockIdx.x];
  const PGraph& G = gs[t & 0xFFFu];
  sub_mean(G.Y, G.n, k, G.part, (G.n + 255) / 256, (size_t)(t >> 12) * blockDim.x + threadIdx.x);
}

}  // namespace

int project_panel(cdl_ctx* ctx, const double* panel, int64_t n64, int r0, int rows, int k, uint64_t seed,
                  double* Y, const unsigned long long* amax_bits) {
  const int n = (int)n64;
  const int W = (k + 31) / 32;
  const int rpb = std::max(1, std::min(MAX_RPB, 256 / (2 * W)));
  const int threads = rpb * 2 * W;
  const size_t smem = project_smem_bytes(rpb, W);
  const int r1 = std::min(n, r0 + rows);
  const int blocks = (r1 - r0 + rpb - 1) / rpb;
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_project_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  if (blocks <= 0) return CDL_OK;
  Launch L(ctx, CDL_KC_PROJECT, (double)(r1 - r0) * (n - 1) * k);
  k_project_panel<<<blocks, threads, smem, ctx->stream>>>(panel, n, k, W, rpb, (uint32_t)(seed & 0xffffffffu),
                                                          (uint32_t)(seed >> 32), 1.0 / std::sqrt((double)k), Y,
                                                          amax_bits, r0, r1);
  return L.done();
}

// Y -= column means (the exact Y has zero column sums), over all n rows.
int project_center(cdl_ctx* ctx, int64_t n64, int k, double* Y) {
  const int n = (int)n64;
  const int nparts = (n + 255) / 256;
  void* vpart;
  CDL_TRY(ws_get(ctx, "project.colsum", (size_t)(nparts + 1) * k * sizeof(double), &vpart));
  double* part = static_cast<double*>(vpart);
  double* mean = part + (size_t)nparts * k;
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_colsum<<<nparts, 256, 0, ctx->stream>>>(Y, n, k, part);
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_col_mean<<<(k + 255) / 256, 256, 0, ctx->stream>>>(part, nparts, n, k, mean);
    CDL_TRY(L.done());
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_sub_mean<<<(unsigned)(((size_t)n * k + 255) / 256), 256, 0, ctx->stream>>>(Y, n, k, mean);
  return L.done();
}

int project(cdl_ctx* ctx, const double* A, int64_t n64, int k, uint64_t seed, double* Y,
            const unsigned long long* amax_bits) {
  const int n = (int)n64;
  const int W = (k + 31) / 32;
  const int rpb = std::max(1, std::min(MAX_RPB, 256 / (2 * W)));
  const int threads = rpb * 2 * W;
  const size_t smem = project_smem_bytes(rpb, W);
  const int blocks = (n + rpb - 1) / rpb;
  const double scale = 1.0 / std::sqrt((double)k);
  // One split per 4096-edge chunk, so that small row counts still fill the
  // GPU in many waves; past 2 GB of partial sums (n above about 90k at
  // k = 128) the row blocks alone are plenty and one split is used.
  int nsplit = (n + CHUNK - 1) / CHUNK;
  if ((double)nsplit * n * k * sizeof(double) > 2147483648.0) nsplit = 1;
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  const void* vmax = amax_bits;
  if (!vmax) {
    void* w;
    CDL_TRY(ws_get(ctx, "project.amax", sizeof(unsigned long long), &w));
    CDL_TRY(abs_max_bits(ctx, A, (size_t)n * n, static_cast<unsigned long long*>(w)));
    vmax = w;
  }
  double* out = Y;
  if (nsplit > 1) {
    void* vp;
    CDL_TRY(ws_get(ctx, "project.partial", (size_t)nsplit * n * k * sizeof(double), &vp));
    out = static_cast<double*>(vp);
  }
  {
    Launch L(ctx, CDL_KC_PROJECT, (double)n * (n - 1) * k);
    k_project<<<dim3(blocks, nsplit), threads, smem, ctx->stream>>>(A, n, k, W, rpb, (uint32_t)(seed & 0xffffffffu),
                                                                    (uint32_t)(seed >> 32), scale, out,
                                                                    static_cast<const unsigned long long*>(vmax));
    CDL_TRY(L.done());
  }
  if (nsplit > 1) {
    const size_t cnt = (size_t)n * k;
    Launch L(ctx, CDL_KC_MISC, 0);
    k_project_sum<<<(unsigned)std::min<size_t>((cnt + 255) / 256, (size_t)ctx->sm_count * 8), 256, 0, ctx->stream>>>(
        out, nsplit, cnt, scale, Y);
    CDL_TRY(L.done());
  }
  return project_center(ctx, n, k, Y);
}

int project_rows_per_block(int k) {
  const int W = (k + 31) / 32;
  return std::max(1, std::min(MAX_RPB, 256 / (2 * W)));
}

int project_grouped(cdl_ctx* ctx, const PGraph* gs, int G2, BTiles blocks, int rpb, int k, uint64_t seed,
                    BTiles chunks, BTiles elem, double adds) {
  const int W = (k + 31) / 32;
  if (rpb < 1 || rpb > project_rows_per_block(k)) return CDL_ERR_INVALID_ARG;
  const int threads = rpb * 2 * W;
  const size_t smem = project_smem_bytes(rpb, W);
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_g_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  (void)G2;
  {
    Launch L(ctx, CDL_KC_PROJECT, adds);
    k_g_project<<<blocks.count, threads, smem, ctx->stream>>>(blocks.p, gs, k, W, rpb, (uint32_t)(seed & 0xffffffffu),
                                                              (uint32_t)(seed >> 32), 1.0 / std::sqrt((double)k));
    CDL_TRY(L.done());
  }
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_g_colsum<<<chunks.count, 256, 0, ctx->stream>>>(chunks.p, gs, k);
    CDL_TRY(L.done());
  }
  Launch L(ctx, CDL_KC_MISC, 0);
  k_g_sub_mean<<<elem.count, 256, 0, ctx->stream>>>(elem.p, gs, k);
  return L.done();
}

}  // namespace cdl
