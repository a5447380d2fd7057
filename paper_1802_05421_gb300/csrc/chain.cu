// Inverse chain (Alg. 2, ChainProduct) on CUDA cores: the deflated level-0
// formation used by every precision, the float32/float64 symmetric squaring
// S~_{i+1} = S~_i^2 and the chain-apply products S~_i x of the solve.
//
// Deflation: S = D^{-1/2} A D^{-1/2} has eigenvalue 1 with unit eigenvector
// u = D^{1/2} 1 / sqrt(vol). S~ = S - u u^T satisfies S~^{2^i} = S^{2^i} - u u^T
// (u is orthogonal to the other eigenvectors), so the squarings of S~ give the
// chain levels minus the u u^T part. The solve only applies the levels to
// D^{-1/2} b with b orthogonal to 1, i.e. to vectors orthogonal to u, where
// both act identically; without the eigenvalue 1 rounding errors are not
// amplified by the repeated squaring.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "ff.cuh"
#include "internal.h"
#include "tiles.cuh"

namespace cdl {
namespace {

// rsqrt_d_i = D_i^{-1/2}, u_i = (D_i / vol)^{1/2}; zero in the padding.
// Float copies rsf, uf feed the bf16 level-0 pass.
__device__ __forceinline__ void chain_vector(const double* __restrict__ D, const double* __restrict__ vol, int n,
                                             double* __restrict__ rsd, double* __restrict__ u,
                                             float* __restrict__ rsf, float* __restrict__ uf, int i) {
  if (i < n) {
    double di = D[i];
    rsd[i] = 1.0 / sqrt(di);
    u[i] = sqrt(di / *vol);
  } else {
    rsd[i] = 0.0;
    u[i] = 0.0;
  }
  rsf[i] = (float)rsd[i];
  uf[i] = (float)u[i];
}

__global__ void k_chain_vectors(const double* __restrict__ D, const double* __restrict__ vol,
                                int n, int npad, double* __restrict__ rsd, double* __restrict__ u,
                                float* __restrict__ rsf, float* __restrict__ uf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) chain_vector(D, vol, n, rsd, u, rsf, uf, i);
}

template <typename T>
__device__ __forceinline__ T to_level(double v);
template <>
__device__ __forceinline__ double to_level<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_level<float>(double v) { return (float)v; }

// S~_0[i][j] = A_ij (rsd_i rsd_j) - u_i u_j (float64 arithmetic, each product
// formed symmetrically in i and j so the level is exactly symmetric), zero padded.
template <typename T>
__global__ void __launch_bounds__(256) k_chain_init(const double* __restrict__ A, int n, int npad,
                                                     const double* __restrict__ rsd,
                                                     const double* __restrict__ u, T* __restrict__ L0) {
  for (int i = blockIdx.x; i < npad; i += gridDim.x) {
    T* out = L0 + (size_t)i * npad;
    if (i >= n) {
      for (int j = threadIdx.x; j < npad; j += blockDim.x) out[j] = to_level<T>(0.0);
      continue;
    }
    const double ri = rsd[i], ui = u[i];
    const double* row = A + (size_t)i * n;
    for (int j = threadIdx.x; j < npad; j += blockDim.x) {
      double v = 0.0;
      if (j < n) v = row[j] * (ri * rsd[j]) - ui * u[j];
      out[j] = to_level<T>(v);
    }
  }
}

// ---- fp8 (e4m3) chains: level i stores value / s_i with s_i = amax_i / 448,
// amax_i a bound on |value| (float bits, so atomicMax on the bits orders them).

__device__ __forceinline__ float fp8_scale_of(unsigned amax_bits) {
  const float a = __uint_as_float(amax_bits);
  return a > 0.f ? a * (1.0f / 448.0f) : 1.0f;
}

// amax_0 = max |level 0| over the bf16 level.
__global__ void __launch_bounds__(256) k_absmax_bf16(const __nv_bfloat16* __restrict__ L, size_t count,
                                                      unsigned* __restrict__ amax) {
  float m = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(__bfloat162float(L[i])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

// level 0 in e4m3 from its bf16 copy.
__global__ void __launch_bounds__(256) k_quant_fp8(const __nv_bfloat16* __restrict__ L, size_t count,
                                                    const unsigned* __restrict__ amax, uint8_t* __restrict__ Q) {
  const float inv = 1.0f / fp8_scale_of(*amax);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    Q[i] = (uint8_t)__nv_cvt_float_to_fp8(__bfloat162float(L[i]) * inv, __NV_SATFINITE, __NV_E4M3);
}

// amax_{i+1} = (1 + 2^-16) max_r sum_c (s_i q_rc)^2: for the symmetric level S,
// |(S S)_ab| <= |row a| |row b| <= max_r |row r|^2, attained on the diagonal,
// so the bound is tight and the squaring's output never overflows e4m3.
__global__ void __launch_bounds__(256) k_rownorm_fp8(const uint8_t* __restrict__ Q, int npad,
                                                      const unsigned* __restrict__ amax_in,
                                                      unsigned* __restrict__ amax_out) {
  __shared__ float red[8];
  const float s = fp8_scale_of(*amax_in);
  float m = 0.f;
  for (int r = blockIdx.x; r < npad; r += gridDim.x) {
    const uint8_t* row = Q + (size_t)r * npad;
    float acc = 0.f;
    for (int c = threadIdx.x * 4; c < npad; c += blockDim.x * 4) {
      const uint32_t w = *reinterpret_cast<const uint32_t*>(row + c);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        __nv_fp8_e4m3 q;
        q.__x = (__nv_fp8_storage_t)((w >> (8 * b)) & 0xFFu);
        const float v = (float)q;
        acc = __fmaf_rn(v, v, acc);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < 8; ++w) t += red[w];
      m = fmaxf(m, t * s * s);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(amax_out, __float_as_uint(m * (1.0f + 0x1p-16f)));
}

// A as float hi + lo planes for the float-float residual (integer split).
__global__ void __launch_bounds__(256) k_split_a(const double* __restrict__ A, size_t count,
                                                  float* __restrict__ hi, float* __restrict__ lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const ff v = split_nonneg(A[i]);
    hi[i] = v.hi;
    lo[i] = v.lo;
  }
}

// max |x_i| as float64 bits (for x >= 0 the bit patterns order like the values).
__global__ void __launch_bounds__(256) k_abs_max_bits(const double* __restrict__ x, size_t count,
                                                       unsigned long long* __restrict__ out) {
  unsigned long long m = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull;
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// A / 2^s on the grid 2^-48 as the integer N = round(A 2^(48 - s)), with 2^s
// the least power of two (s >= 0) not below max A, so that A / 2^s lies in
// [0, 1] (the kernel graphs have s = 0). The rounding uses the float64 bit
// pattern (integer operations only): A = m 2^(e - 52), N = m / 2^(4 - e + s)
// rounded to nearest (ties up).
__device__ __forceinline__ long long grid48(double a, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;                                   // zero (no subnormal kernel values)
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = 1023 + 4 - e + s;                         // a = m 2^(e - 1075); a 2^(48 - s) = m 2^(e - 1027 - s)
  if (sh >= 60) return 0;
  if (sh <= 0) return (long long)(m << -sh);
  return (long long)((m + (1ull << (sh - 1))) >> sh);
}


// Tensor chains: level 0 in bf16, A_ij (rf_i rf_j) - uf_i uf_j formed in
// float32 with float copies of D^{-1/2} and u (the float32 error, a few 1e-7
// relative to either product, is far below the bf16 rounding of the result);
// A as two bf16 matrices A_hi + A_lo (the operand of the solve's recursive
// residual update); and A / 2^s as six exact bf16 digit planes (N of grid48
// split into signed base-256 digits d_t, plane t holding d_t 2^-8t), the
// operand of its full residual; all in one pass over A; padding rows
// and columns zero. Conversions avoid the float64 pipe (the scarce one): the
// float of A_ij rounded to nearest by integer operations, the digits bottom-up
// (balanced base 256 on two 24-bit halves of N = A_ij 2^(48-s)) and their bf16
// bit patterns by exact float32 arithmetic (digits6_fbits).
__device__ __forceinline__ float d2f_rn_nonneg(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126) return 0.f;                               // below the float normal range
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  unsigned q = (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull), half = 1u << 28;
  if (rem > half || (rem == half && (q & 1u))) ++q;
  if (q >> 23) {
    q = 0;
    ++e;
  }
  return __uint_as_float(((unsigned)(e + 127) << 23) | q);
}

// The six signed base-256 digits of N (N in [0, 2^48]) as float32 bit
// patterns of d_t 2^-8(t+1), computed bottom-up on two 24-bit halves of N
// (the five lower digits in [-128, 128), the leading one in [0, 256]). Each
// digit is formed exactly without a conversion instruction: with u = (v + 128)
// mod 256, the float 2^23 + u (bit pattern 0x4B000000 | u) times 2^-8(t+1)
// minus (2^23 + 128) 2^-8(t+1) is (u - 128) 2^-8(t+1) = d_t 2^-8(t+1), exact
// in one fused multiply-add; the next v is (v + 128) >> 8. |d_t| <= 256 has at
// most 8 significant bits, so the upper 16 bits of each pattern are the bf16
// of the digit, exactly.
template <int T>
__device__ __forceinline__ uint32_t digit_fbits(int& v) {
  constexpr float sc = (float)(1.0 / (double)(1ull << (8 * (T + 1))));
  const int t = v + 128;
  v = t >> 8;
  return __float_as_uint(__fmaf_rn(__uint_as_float(0x4B000000u | (uint32_t)(t & 255)), sc, -8388736.0f * sc));
}

__device__ __forceinline__ void digits6_fbits(long long N, uint32_t (&f)[6]) {
  int lo = (int)(N & 0xFFFFFF), hi = (int)(N >> 24);
  f[5] = digit_fbits<5>(lo);
  f[4] = digit_fbits<4>(lo);
  f[3] = digit_fbits<3>(lo);
  hi += lo;                                               // carry of the lower half
  f[2] = digit_fbits<2>(hi);
  f[1] = digit_fbits<1>(hi);
  constexpr float sc0 = 1.0f / 256.0f;                    // leading digit hi in [0, 256]
  f[0] = __float_as_uint(__fmaf_rn(__uint_as_float(0x4B000000u | (uint32_t)hi), sc0, -8388608.0f * sc0));
}

// SL = false (the batched form's chains, which keep no slices): S and
// a_scale are not touched (they may be null).
// One group of 8 columns (index g over the npad x npad / 8 groups, row-major)
// of k_chain_init_tc's outputs.
template <bool SL>
__device__ __forceinline__ void chain_init_tc_group(const double* __restrict__ A, int n, int npad,
                                                    const float* __restrict__ rsf, const float* __restrict__ uf,
                                                    __nv_bfloat16* __restrict__ L0, __nv_bfloat16* __restrict__ Ahi,
                                                    __nv_bfloat16* __restrict__ Alo, uint16_t* __restrict__ S, int sexp,
                                                    size_t g) {
  const size_t plane = (size_t)npad * npad;
  const int gpr = npad / 8;                               // groups of 8 columns per row
  {
    const int i = (int)(g / gpr), j0 = (int)(g % gpr) * 8;
    const size_t o = (size_t)i * npad + j0;
    uint32_t wl[4] = {0, 0, 0, 0}, wh[4] = {0, 0, 0, 0}, wo[4] = {0, 0, 0, 0}, ws[6][4] = {};
    if (i < n) {
      const float ri = rsf[i], ui = uf[i];
      const double* row = A + (size_t)i * n;
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float v[2] = {0.f, 0.f}, af[2] = {0.f, 0.f};
        uint32_t dg[2][6] = {};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = j0 + e + h;
          if (j < n) {
            const double a = row[j];
            af[h] = d2f_rn_nonneg(a);
            v[h] = __fmaf_rn(af[h], __fmul_rn(ri, rsf[j]), -__fmul_rn(ui, uf[j]));
            if constexpr (SL) digits6_fbits(grid48(a, sexp), dg[h]);
          }
        }
        const __nv_bfloat162 lv = __floats2bfloat162_rn(v[0], v[1]);
        const __nv_bfloat162 hv = __floats2bfloat162_rn(af[0], af[1]);
        const float2 hf = __bfloat1622float2(hv);
        const __nv_bfloat162 ov = __floats2bfloat162_rn(__fsub_rn(af[0], hf.x), __fsub_rn(af[1], hf.y));
        wl[e / 2] = *reinterpret_cast<const uint32_t*>(&lv);
        wh[e / 2] = *reinterpret_cast<const uint32_t*>(&hv);
        wo[e / 2] = *reinterpret_cast<const uint32_t*>(&ov);
        if constexpr (SL) {
#pragma unroll
          for (int t = 0; t < 6; ++t)
            ws[t][e / 2] = __byte_perm(dg[0][t], dg[1][t], 0x7632);   // upper halves: the two bf16 digits
        }
      }
    }
    *reinterpret_cast<uint4*>(L0 + o) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    *reinterpret_cast<uint4*>(Ahi + o) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4*>(Alo + o) = make_uint4(wo[0], wo[1], wo[2], wo[3]);
    if constexpr (SL) {
#pragma unroll
      for (int t = 0; t < 6; ++t)
        *reinterpret_cast<uint4*>(S + (size_t)t * plane + o) = make_uint4(ws[t][0], ws[t][1], ws[t][2], ws[t][3]);
    }
  }
}

template <bool SL>
__global__ void __launch_bounds__(256) k_chain_init_tc(const double* __restrict__ A, int n, int npad,
                                                        const float* __restrict__ rsf, const float* __restrict__ uf,
                                                        __nv_bfloat16* __restrict__ L0, __nv_bfloat16* __restrict__ Ahi,
                                                        __nv_bfloat16* __restrict__ Alo, uint16_t* __restrict__ S,
                                                        double* __restrict__ a_scale) {
  int sexp = 0;
  if constexpr (SL) {
    sexp = pow2_exp_above((unsigned long long)__double_as_longlong(a_scale[1]));
    if (blockIdx.x == 0 && threadIdx.x == 0) a_scale[0] = __longlong_as_double((long long)(1023 + sexp) << 52);
  }
  const int gpr = npad / 8;                               // groups of 8 columns per row
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)npad * gpr;
       g += (size_t)gridDim.x * blockDim.x)
    chain_init_tc_group<SL>(A, n, npad, rsf, uf, L0, Ahi, Alo, S, sexp, g);
}


// C = P^T Q on CUDA cores: C[m][c] = sum_k P[k][m] Q[k][c]; P is K x M and Q
// is K x N, both row-major, so both tiles are contiguous k-major slabs.
// SYM: P == Q == S symmetric, M == N; only tiles bi <= bj are computed and
//      each is also written transposed (C = S^2 is symmetric).
// Otherwise: split-K partial products, C + split * M * ldc.
template <typename T, int BM, int BN, int BK, int TM, int TN, bool SYM>
__global__ void __launch_bounds__(256) k_gemm_tn(const T* __restrict__ P, int ldp,
                                                  const T* __restrict__ Q, int ldq, T* __restrict__ C,
                                                  int ldc, int M, int N, int kchunk) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN];
  int m0, c0, k0, k1;
  bool mirror = false;
  if (SYM) {
    int bi, bj;
    tri_index(blockIdx.x, M / BM, bi, bj);
    m0 = bi * BM;
    c0 = bj * BN;
    mirror = bi != bj;
    k0 = 0;
    k1 = kchunk;
  } else {
    m0 = blockIdx.x * BM;
    c0 = blockIdx.y * BN;
    k0 = blockIdx.z * kchunk;
    k1 = k0 + kchunk;
    C += (size_t)blockIdx.z * M * ldc;
  }
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  constexpr int A_LD = BM * BK / 256;   // elements each thread loads per tile
  constexpr int B_LD = BN * BK / 256;
  T ra[A_LD], rb[B_LD];
  auto gload = [&](int kt) {
#pragma unroll
    for (int e = 0; e < A_LD; ++e) {
      int idx = tid + e * 256;
      int kk = idx / BM, mm = idx % BM;
      ra[e] = P[(size_t)(kt + kk) * ldp + m0 + mm];
    }
#pragma unroll
    for (int e = 0; e < B_LD; ++e) {
      int idx = tid + e * 256;
      int kk = idx / BN, cc = idx % BN;
      int c = c0 + cc;
      rb[e] = (c < N) ? Q[(size_t)(kt + kk) * ldq + c] : T(0);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int e = 0; e < A_LD; ++e) {
      int idx = tid + e * 256;
      As[buf][idx / BM][idx % BM] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < B_LD; ++e) {
      int idx = tid + e * 256;
      Bs[buf][idx / BN][idx % BN] = rb[e];
    }
  };
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
  gload(k0);
  sstore(0);
  __syncthreads();
  int buf = 0;
  for (int kt = k0; kt < k1; kt += BK) {
    const bool more = kt + BK < k1;
    if (more) gload(kt + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM / 2; ++a) {
        av[a] = As[buf][kk][ty * (TM / 2) + a];
        av[TM / 2 + a] = As[buf][kk][BM / 2 + ty * (TM / 2) + a];
      }
#pragma unroll
      for (int b = 0; b < TN / 2; ++b) {
        bv[b] = Bs[buf][kk][tx * (TN / 2) + b];
        bv[TN / 2 + b] = Bs[buf][kk][BN / 2 + tx * (TN / 2) + b];
      }
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    if (more) {
      sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    int m = m0 + (a < TM / 2 ? ty * (TM / 2) + a : BM / 2 + ty * (TM / 2) + a - TM / 2);
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      int c = c0 + (b < TN / 2 ? tx * (TN / 2) + b : BN / 2 + tx * (TN / 2) + b - TN / 2);
      if (c < N) {
        C[(size_t)m * ldc + c] = acc[a][b];
        if (SYM && mirror) C[(size_t)c * ldc + m] = acc[a][b];
      }
    }
  }
}

template <typename T>
int square_impl(cdl_ctx* ctx, cdl_chain* ch, int level) {
  const int np = (int)ch->npad;
  const T* S = static_cast<const T*>(ch->level(level));
  T* C = static_cast<T*>(ch->level(level + 1));
  const double flops = (double)ch->n * ch->n * (ch->n + 1.0);   // symmetric product
  if constexpr (sizeof(T) == 4) {
    constexpr int B = 128;
    const int nb = np / B;
    Launch L(ctx, CDL_KC_SQUARE, flops);
    k_gemm_tn<T, B, B, 8, 8, 8, true><<<nb * (nb + 1) / 2, 256, 0, ctx->stream>>>(S, np, S, np, C, np, np, np, np);
    return L.done();
  } else {
    constexpr int B = 64;
    const int nb = np / B;
    Launch L(ctx, CDL_KC_SQUARE, flops);
    k_gemm_tn<T, B, B, 8, 4, 4, true><<<nb * (nb + 1) / 2, 256, 0, ctx->stream>>>(S, np, S, np, C, np, np, np, np);
    return L.done();
  }
}


// ---- graphs regenerated in row panels (the pair driver's larger-than-memory form)
// Level-0 rows r0 .. r0 + rows - 1 of a bf16 chain from a panel holding those
// rows of A (A[(i - r0) n + j]): the same arithmetic as k_chain_init_tc, so
// the level equals the one formed from the whole matrix; padding zero.
__global__ void __launch_bounds__(256) k_panel_level0(const double* __restrict__ P, int n, int npad, int r0,
                                                       int rows, const float* __restrict__ rsf,
                                                       const float* __restrict__ uf, __nv_bfloat16* __restrict__ L0) {
  const int gpr = npad / 8;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)rows * gpr;
       g += (size_t)gridDim.x * blockDim.x) {
    const int i = r0 + (int)(g / gpr), j0 = (int)(g % gpr) * 8;
    uint32_t wl[4] = {0, 0, 0, 0};
    if (i < n) {
      const float ri = rsf[i], ui = uf[i];
      const double* row = P + (size_t)(i - r0) * n;
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float v[2] = {0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = j0 + e + h;
          if (j < n) v[h] = __fmaf_rn(d2f_rn_nonneg(row[j]), __fmul_rn(ri, rsf[j]), -__fmul_rn(ui, uf[j]));
        }
        const __nv_bfloat162 lv = __floats2bfloat162_rn(v[0], v[1]);
        wl[e / 2] = *reinterpret_cast<const uint32_t*>(&lv);
      }
    }
    *reinterpret_cast<uint4*>(L0 + (size_t)i * npad + j0) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
  }
}

// The six exact bf16 slices (grid48 with s = 0: Gaussian-kernel graphs have
// A <= 1) of a panel of A holding rows r0 .. r0 + rows - 1 (A[(i - r0) n + j]),
// transposed: plane t, row i, column c holds digit t of A[r0 + c][i] = A[i][r0 + c]
// (A is symmetric), so each row i of a plane is a K-major operand row over the
// panel's columns. Planes are npad x P; zero for i >= n or c >= rows. 32 x 32
// tiles through shared memory: read along i, written along c.
__global__ void __launch_bounds__(256) k_panel_slices_t(const double* __restrict__ P, int n, int npad, int r0,
                                                         int rows, int Pw, uint16_t* __restrict__ S) {
  __shared__ double tile[32][33];
  const int ntc = Pw / 32, nti = npad / 32;
  const size_t plane = (size_t)npad * Pw;
  for (long long t = blockIdx.x; t < (long long)ntc * nti; t += gridDim.x) {
    const int c0 = (int)(t % ntc) * 32, i0 = (int)(t / ntc) * 32;
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int cc = e / 32, ii = e % 32;                   // panel row c0 + cc, column i0 + ii
      const int c = c0 + cc, i = i0 + ii;
      tile[cc][ii] = (c < rows && r0 + c < n && i < n) ? P[(size_t)c * n + i] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int ii = e / 32, cc = e % 32;                   // output row i0 + ii, column c0 + cc
      uint32_t dg[6];
      digits6_fbits(grid48(tile[cc][ii], 0), dg);
      const size_t o = (size_t)(i0 + ii) * Pw + c0 + cc;
#pragma unroll
      for (int q = 0; q < 6; ++q) S[(size_t)q * plane + o] = (uint16_t)(dg[q] >> 16);
    }
  }
}

// ---- batched form: level 0 of every graph in three launches
__global__ void __launch_bounds__(256) k_g_chain_vectors(const uint32_t* __restrict__ tiles,
                                                          const CGraph* __restrict__ cg) {
  const uint32_t t = tiles[blockIdx.x];
  const CGraph& G = cg[t & 0xFFFu];
  const int i = (int)(t >> 12) * 256 + threadIdx.x;
  if (i < G.npad) chain_vector(G.D, G.vol, G.n, G.rsd, G.u, G.rsf, G.uf, i);
}

__global__ void __launch_bounds__(256) k_g_chain_init(const uint32_t* __restrict__ tiles, const CGraph* __restrict__ cg) {
  const uint32_t t = tiles[blockIdx.x];
  const CGraph& G = cg[t & 0xFFFu];
  const size_t groups = (size_t)G.npad * (G.npad / 8);
  const size_t g1 = min(groups, ((size_t)(t >> 12) + 1) * 2048);
  __nv_bfloat16* L0 = static_cast<__nv_bfloat16*>(G.L0);
  __nv_bfloat16* ahi = static_cast<__nv_bfloat16*>(G.aop);
  __nv_bfloat16* alo = ahi + (size_t)G.npad * G.npad;
  // the exact slices of A on the grids 2^-8s (kernel weights are at most 1: scale 2^0)
  for (size_t g = (size_t)(t >> 12) * 2048 + threadIdx.x; g < g1; g += 256)
    chain_init_tc_group<true>(G.A, G.n, G.npad, G.rsf, G.uf, L0, ahi, alo, G.aslices, 0, g);
}
}  // namespace

int abs_max_bits(cdl_ctx* ctx, const double* x, size_t count, unsigned long long* out) {
  CDL_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned long long), ctx->stream));
  Launch L(ctx, CDL_KC_MISC, 8.0 * (double)count);
  const size_t blocks = std::min<size_t>((count + 255) / 256, (size_t)ctx->sm_count * 8);
  k_abs_max_bits<<<(unsigned)std::max<size_t>(blocks, 1), 256, 0, ctx->stream>>>(x, count, out);
  return L.done();
}

int chain_init(cdl_ctx* ctx, cdl_chain* ch, const double* A) {
  const int n = (int)ch->n, np = (int)ch->npad;
  if (ch->ahl) {
    const size_t cnt = (size_t)n * n;
    Launch L(ctx, CDL_KC_CHAIN_INIT, 16.0 * cnt);
    k_split_a<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(A, cnt, ch->ahl, ch->ahl + cnt);
    CDL_TRY(L.done());
  }
  if (ch->aslices) {   // the slices' scale: max A, known before level 0 is formed
    unsigned long long* mb = reinterpret_cast<unsigned long long*>(ch->a_scale + 1);
    if (ctx->amax_hint_A == A && ctx->amax_hint_bits)
      CDL_CUDA_TRY(cudaMemcpyAsync(mb, ctx->amax_hint_bits, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    else
      CDL_TRY(abs_max_bits(ctx, A, (size_t)n * n, mb));
  }
  ctx->amax_hint_A = nullptr;
  ctx->amax_hint_bits = nullptr;
  void* wsu;
  CDL_TRY(ws_get(ctx, "chain.u", (size_t)np * (sizeof(double) + 2 * sizeof(float)), &wsu));
  double* u = static_cast<double*>(wsu);
  float* rsf = reinterpret_cast<float*>(u + np);
  float* uf = rsf + np;
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_chain_vectors<<<(np + 255) / 256, 256, 0, ctx->stream>>>(ch->D, ch->vol, n, np, ch->rsqrt_d, u, rsf, uf);
    CDL_TRY(L.done());
  }
  const bool tensor = ch->aslices != nullptr;
  // algorithmic bytes: A read once; level 0 written (plus A hi, lo and, for
  // single-graph tensor chains, six slices)
  const double bytes = 8.0 * n * (double)n + (double)ch->elem * np * (double)np +
                       (ch->aop ? 4.0 * np * (double)np : 0.0) + (tensor ? 12.0 * np * (double)np : 0.0);
  const int blocks = std::min(np, ctx->sm_count * 8);
  // level 0 in bf16 with A hi/lo and the slices (tensor chains)
  auto init16 = [&](void* L0) {
    __nv_bfloat16* l0 = static_cast<__nv_bfloat16*>(L0);
    __nv_bfloat16* ahi = static_cast<__nv_bfloat16*>(ch->aop);
    __nv_bfloat16* alo = ahi + (size_t)np * np;
    if (tensor)
      k_chain_init_tc<true><<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(
          A, n, np, rsf, uf, l0, ahi, alo, static_cast<uint16_t*>(ch->aslices), ch->a_scale);
    else
      k_chain_init_tc<false><<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(A, n, np, rsf, uf, l0, ahi, alo, nullptr,
                                                                         nullptr);
  };
  Launch L(ctx, CDL_KC_CHAIN_INIT, bytes);
  switch (ch->dtype) {
    case CDL_F64:
      k_chain_init<double><<<blocks, 256, 0, ctx->stream>>>(A, n, np, ch->rsqrt_d, u,
                                                            static_cast<double*>(ch->level(0)));
      break;
    case CDL_F32:
      k_chain_init<float><<<blocks, 256, 0, ctx->stream>>>(A, n, np, ch->rsqrt_d, u,
                                                           static_cast<float*>(ch->level(0)));
      break;
    case CDL_FP8E4M3: {
      // bf16 level 0 (apply copy) and A_hi/A_lo, then the bound and the e4m3 level
      CDL_CUDA_TRY(cudaMemsetAsync(ch->amax, 0, ch->d * sizeof(unsigned), ctx->stream));
      init16(ch->level16(0));
      CDL_TRY(L.done());
      const size_t cnt = (size_t)np * np;
      {
        Launch L2(ctx, CDL_KC_CHAIN_INIT, 2.0 * cnt);
        k_absmax_bf16<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(
            static_cast<const __nv_bfloat16*>(ch->level16(0)), cnt, ch->amax);
        CDL_TRY(L2.done());
      }
      Launch L3(ctx, CDL_KC_CHAIN_INIT, 3.0 * cnt);
      k_quant_fp8<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(static_cast<const __nv_bfloat16*>(ch->level16(0)),
                                                              cnt, ch->amax, static_cast<uint8_t*>(ch->level(0)));
      return L3.done();
    }
    case CDL_FP8E4M3_T128:
      init16(ch->level16(0));
      CDL_TRY(L.done());
      return fp8t_quantize_level0(ctx, ch);
    case CDL_BF16: {
      void* L0 = ch->host_levels ? ooc_write_begin(ctx, ch, 0) : ch->level(0);
      init16(L0);
      CDL_TRY(L.done());
      return ch->host_levels ? ooc_write_end(ctx, ch, 0) : CDL_OK;
    }
    default:
      return CDL_ERR_UNSUPPORTED;
  }
  return L.done();
}

// Max absolute row sum of an npad x npad level (rows of threads; atomicMax
// on the bits of non-negative floats orders them like their values).
template <typename T>
__global__ void __launch_bounds__(256) k_level_inf_norm(const T* __restrict__ L, int np, unsigned* __restrict__ out) {
  __shared__ float red[8];
  for (int i = blockIdx.x; i < np; i += gridDim.x) {
    float s = 0.f;
    const T* row = L + (size_t)i * np;
    for (int j = threadIdx.x; j < np; j += 256) s += fabsf((float)row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < 8; ++w) t += red[w];
      atomicMax(out, __float_as_uint(t * (1.0f + 0x1p-12f)));   // rounded up: a bound
    }
    __syncthreads();
  }
}

int level_inf_norm(cdl_ctx* ctx, const cdl_chain* ch, int level, unsigned* out_bits) {
  const int np = (int)ch->npad;
  const int blocks = std::min(np, ctx->sm_count * 8);
  CDL_CUDA_TRY(cudaMemsetAsync(out_bits, 0, sizeof(unsigned), ctx->stream));
  Launch L(ctx, CDL_KC_MISC, 2.0 * np * (double)np);
  switch (ch->dtype) {
    case CDL_F64:
      k_level_inf_norm<double><<<blocks, 256, 0, ctx->stream>>>(static_cast<const double*>(ch->level(level)), np,
                                                                out_bits);
      break;
    case CDL_F32:
      k_level_inf_norm<float><<<blocks, 256, 0, ctx->stream>>>(static_cast<const float*>(ch->level(level)), np,
                                                               out_bits);
      break;
    default:   // bf16 levels, or the bf16 copies of e4m3 levels
      if (ch->host_levels) return CDL_ERR_UNSUPPORTED;
      k_level_inf_norm<__nv_bfloat16><<<blocks, 256, 0, ctx->stream>>>(
          static_cast<const __nv_bfloat16*>(ch->level16(level)), np, out_bits);
      break;
  }
  return L.done();
}

int fp8_level_bound(cdl_ctx* ctx, cdl_chain* ch, int level) {
  const int np = (int)ch->npad;
  Launch L(ctx, CDL_KC_MISC, (double)np * np);
  k_rownorm_fp8<<<std::min(np, ctx->sm_count * 8), 256, 0, ctx->stream>>>(
      static_cast<const uint8_t*>(ch->level(level)), np, ch->amax + level, ch->amax + level + 1);
  return L.done();
}

int chain_square_simt(cdl_ctx* ctx, cdl_chain* ch, int level) {
  if (ch->dtype == CDL_F32) return square_impl<float>(ctx, ch, level);
  if (ch->dtype == CDL_F64) return square_impl<double>(ctx, ch, level);
  return CDL_ERR_UNSUPPORTED;
}

// partial[s] = (level_i)^T x restricted to k-range s (level_i is symmetric, so
// this is level_i x). x: npad x kp row-major in the chain's dtype.
int apply_simt(cdl_ctx* ctx, const cdl_chain* ch, int level, const void* x, void* partial, int kp,
               int splits) {
  const int np = (int)ch->npad;
  const int kchunk = np / splits;
  const double bytes = (double)ch->elem * np * (double)np;
  if (ch->dtype == CDL_F32) {
    constexpr int BM = 128, BN = 64;
    dim3 grid(np / BM, (kp + BN - 1) / BN, splits);
    Launch L(ctx, CDL_KC_APPLY, bytes);
    k_gemm_tn<float, BM, BN, 8, 8, 4, false><<<grid, 256, 0, ctx->stream>>>(
        static_cast<const float*>(ch->level(level)), np, static_cast<const float*>(x), kp,
        static_cast<float*>(partial), kp, np, kp, kchunk);
    return L.done();
  }
  if (ch->dtype == CDL_F64) {
    constexpr int BM = 64, BN = 64;
    dim3 grid(np / BM, (kp + BN - 1) / BN, splits);
    Launch L(ctx, CDL_KC_APPLY, bytes);
    k_gemm_tn<double, BM, BN, 8, 4, 4, false><<<grid, 256, 0, ctx->stream>>>(
        static_cast<const double*>(ch->level(level)), np, static_cast<const double*>(x), kp,
        static_cast<double*>(partial), kp, np, kp, kchunk);
    return L.done();
  }
  return CDL_ERR_UNSUPPORTED;
}


// Chain vectors (D^{-1/2}, u and their float copies) from the chain's D and
// vol, for a chain whose level 0 is formed panel by panel.
int chain_vectors_only(cdl_ctx* ctx, cdl_chain* ch) {
  const int n = (int)ch->n, np = (int)ch->npad;
  void* wsu;
  CDL_TRY(ws_get(ctx, "chain.u", (size_t)np * (sizeof(double) + 2 * sizeof(float)), &wsu));
  double* u = static_cast<double*>(wsu);
  float* rsf = reinterpret_cast<float*>(u + np);
  float* uf = rsf + np;
  Launch L(ctx, CDL_KC_MISC, 0);
  k_chain_vectors<<<(np + 255) / 256, 256, 0, ctx->stream>>>(ch->D, ch->vol, n, np, ch->rsqrt_d, u, rsf, uf);
  return L.done();
}

int chain_level0_panel(cdl_ctx* ctx, cdl_chain* ch, void* L0, const double* panel, int r0, int rows) {
  const int n = (int)ch->n, np = (int)ch->npad;
  if (ch->dtype != CDL_BF16 || r0 % 8) return CDL_ERR_UNSUPPORTED;
  void* wsu;
  CDL_TRY(ws_get(ctx, "chain.u", (size_t)np * (sizeof(double) + 2 * sizeof(float)), &wsu));
  const float* rsf = reinterpret_cast<const float*>(static_cast<double*>(wsu) + np);
  const float* uf = rsf + np;
  Launch L(ctx, CDL_KC_CHAIN_INIT, 8.0 * rows * (double)n + 2.0 * rows * (double)np);
  k_panel_level0<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(panel, n, np, r0, rows, rsf, uf,
                                                             static_cast<__nv_bfloat16*>(L0));
  return L.done();
}

int panel_slices_t(cdl_ctx* ctx, const double* panel, int n, int np, int r0, int rows, int Pw, void* slicesT) {
  if (Pw % 32 || np % 32) return CDL_ERR_INVALID_ARG;
  Launch L(ctx, CDL_KC_RESIDUAL, 0);
  k_panel_slices_t<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(panel, n, np, r0, rows, Pw,
                                                               static_cast<uint16_t*>(slicesT));
  return L.done();
}


int chain_init_grouped(cdl_ctx* ctx, const CGraph* cg, BTiles vec, BTiles init, double bytes) {
  {
    Launch L(ctx, CDL_KC_MISC, 0);
    k_g_chain_vectors<<<vec.count, 256, 0, ctx->stream>>>(vec.p, cg);
    CDL_TRY(L.done());
  }
  Launch L(ctx, CDL_KC_CHAIN_INIT, bytes);
  k_g_chain_init<<<init.count, 256, 0, ctx->stream>>>(init.p, cg);
  return L.done();
}

}  // namespace cdl
