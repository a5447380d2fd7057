// Random projection Y = (Q W^{1/2} B)^T of Alg. 1 ("y = W^{1/2} B q") and
// Alg. 3, formed edge by edge without materialising B or Q (the Map +
// ReduceByKey of Sec. 3.3):
//   Y[i, r] = k^{-1/2} sum_{j != i} o_ij s_r(min(i,j), max(i,j)) sqrt(A_ij),
// o_ij = +1 when i < j (i is the head of edge (i, j), Sec. 2), else -1.
// The signs come from Philox4x32-10 (Salmon et al., SC'11) at counter
// (i, j, r / 128, 0) with key (seed low word, seed high word): bit (r mod 32)
// of output word ((r mod 128) / 32) set means +1.
//
// Each thread owns one node row i and 32 projection rows (one Philox word);
// sqrt(A_ij) is formed once per tile in float-float, and the signed sums are
// accumulated in float-float (TwoSum) on the float32 pipes.
#include <cmath>

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

constexpr int JT = 32;   // j-tile

__global__ void __launch_bounds__(256) k_project(const double* __restrict__ A, int n, int k, int W, int rpb,
                                                  uint32_t key0, uint32_t key1, double scale,
                                                  double* __restrict__ Y) {
  extern __shared__ float sm[];
  float* Sh = sm;                    // [rpb][JT]
  float* Sl = sm + rpb * JT;         // [rpb][JT]
  const int t = threadIdx.x;
  const int rl = t / W, w = t % W;
  const int i0 = blockIdx.x * rpb;
  const int i = i0 + rl;
  const bool active = rl < rpb && i < n;
  float ah[32], al[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) ah[b] = al[b] = 0.f;
  for (int j0 = 0; j0 < n; j0 += JT) {
    __syncthreads();
    for (int e = t; e < rpb * JT; e += blockDim.x) {
      const int rr = e / JT, jj = e % JT;
      const int ii = i0 + rr, j = j0 + jj;
      float sh = 0.f, sl = 0.f;
      if (ii < n && j < n) {
        const double a = A[(size_t)ii * n + j];
        const float h = (float)a;
        const float l = (float)(a - (double)h);
        if (h > 0.f) {
          sh = sqrtf(h);
          // sqrt(h + l) = sh + (h - sh^2 + l) / (2 sh) to float-float accuracy
          const float res = __fadd_rn(__fmaf_rn(-sh, sh, h), l);
          sl = res / (2.f * sh);
        }
      }
      Sh[e] = sh;
      Sl[e] = sl;
    }
    __syncthreads();
    if (!active) continue;
    const int jmax = min(JT, n - j0);
    for (int jj = 0; jj < jmax; ++jj) {
      const int j = j0 + jj;
      if (j == i) continue;
      float sh = Sh[rl * JT + jj], sl = Sl[rl * JT + jj];
      if (j < i) {   // i is the tail of edge (j, i)
        sh = -sh;
        sl = -sl;
      }
      const uint32_t lo = (uint32_t)min(i, j), hi = (uint32_t)max(i, j);
      const uint4 o = philox4x32_10(make_uint4(lo, hi, (uint32_t)(w >> 2), 0u), key0, key1);
      const uint32_t wi = w & 3;
      const uint32_t bits = wi == 0 ? o.x : wi == 1 ? o.y : wi == 2 ? o.z : o.w;
      const uint32_t shb = __float_as_uint(sh), slb = __float_as_uint(sl);
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        const uint32_t neg = ((~bits >> b) & 1u) << 31;   // clear bit -> -1
        const float th = __uint_as_float(shb ^ neg);
        const float tl = __uint_as_float(slb ^ neg);
        const float s = __fadd_rn(ah[b], th);
        const float bp = __fsub_rn(s, ah[b]);
        const float err = __fadd_rn(__fsub_rn(ah[b], __fsub_rn(s, bp)), __fsub_rn(th, bp));
        ah[b] = s;
        al[b] = __fadd_rn(al[b], __fadd_rn(err, tl));
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int b = 0; b < 32; ++b) {
    const int r = w * 32 + b;
    if (r < k) Y[(size_t)i * k + r] = ((double)ah[b] + (double)al[b]) * scale;
  }
}

}  // namespace

int project(cdl_ctx* ctx, const double* A, int64_t n64, int k, uint64_t seed, double* Y) {
  const int n = (int)n64;
  const int W = (k + 31) / 32;
  const int rpb = std::max(1, std::min(128, 256 / W));
  const int threads = rpb * W;
  const size_t smem = 2 * (size_t)rpb * JT * sizeof(float);
  const int blocks = (n + rpb - 1) / rpb;
  const double scale = 1.0 / std::sqrt((double)k);
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    attr = true;
  }
  Launch L(ctx, CDL_KC_PROJECT, (double)n * (n - 1) * k);
  k_project<<<blocks, threads, smem, ctx->stream>>>(A, n, k, W, rpb, (uint32_t)(seed & 0xffffffffu),
                                                    (uint32_t)(seed >> 32), scale, Y);
  return L.done();
}

}  // namespace cdl
