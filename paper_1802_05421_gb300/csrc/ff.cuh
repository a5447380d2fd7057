// Float-float ("double-float") arithmetic on the float32 pipes, built from the
// classical error-free transformations: TwoSum (Knuth, TAOCP vol. 2), FastTwoSum
// (Dekker 1971) and TwoProduct through a fused multiply-add. A value is hi + lo
// with |lo| <= ulp(hi)/2, about 48 significant bits. Used where float64-class
// accuracy is needed in O(n^2) work, because float64 runs at about 1/72 of the
// float32 rate on this GPU.
#pragma once

#include <cstdint>

namespace cdl {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Conversions between float and double done with integer operations (the
// float64 pipe also executes the hardware conversions, and it is the scarce
// one on this GPU). f2d_bits is exact for normal floats and zero (subnormal
// floats map to zero); d2f_trunc truncates a double to 24 significant bits
// (exact for the top 24 bits; doubles below the float normal range map to
// zero, beyond it the result is meaningless, callers keep |x| < 2^127).
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long ed = (unsigned long long)(e - 127 + 1023) << 52;
  const unsigned long long m = (unsigned long long)(b & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | ed | m));
}

// Split a float64 x >= 0 into floats hi + lo with hi = x truncated to 24 bits
// and lo the remaining 29 mantissa bits rounded to 24 (|x - hi - lo| <=
// 2^-48 x; below 2^-74, where lo falls under the float normal range, lo is
// subnormal and the bound is 2^-149 absolute), by integer operations and two
// exact scalings. Values below 2^-100 give {0, 0}.
__device__ __forceinline__ ff split_nonneg(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;      // x in [2^e, 2^(e+1))
  if (e < -100) return {0.f, 0.f};
  const uint32_t hi_bits = ((uint32_t)(e + 127) << 23) | ((uint32_t)(b >> 29) & 0x7FFFFFu);
  const uint32_t low29 = (uint32_t)(b & 0x1FFFFFFFull);
  // lo = low29 2^(e - 52) = (low29 2^-52) 2^e: both factors are normal floats
  // for e >= -100 (2^(e - 52) itself is not, below e = -74)
  const float lo = __fmul_rn(__fmul_rn(__uint2float_rn(low29), 0x1p-52f), __uint_as_float((uint32_t)(e + 127) << 23));
  return {__uint_as_float(hi_bits), lo};
}

// The least e >= 0 with x <= 2^e, for the float64 bit pattern of x >= 0
// (zero gives 0).
__device__ __forceinline__ int pow2_exp_above(unsigned long long bits) {
  if (bits == 0) return 0;
  const int e = (int)((bits >> 52) & 0x7FF) - 1023;
  const int up = (bits & 0xFFFFFFFFFFFFFull) != 0 ? e + 1 : e;
  return up > 0 ? up : 0;
}

// Unsigned 64-bit integers to floating point with integer operations only.
// u64_top24: x truncated to its 24 leading bits, as a float (exact for x <
// 2^24). ff_from_u64: x as hi + lo, both truncations (|x - hi - lo| < 2^-47 x).
// u64_to_double_rn: x 2^scale_exp rounded to nearest even, the float64 the
// hardware conversion gives (x 2^scale_exp in the normal range).
__device__ __forceinline__ float u64_top24(unsigned long long x) {
  if (x == 0) return 0.f;
  const int e = 63 - __clzll((long long)x);
  const unsigned long long top = e >= 23 ? (x >> (e - 23)) : (x << (23 - e));
  return __uint_as_float(((uint32_t)(e + 127) << 23) | ((uint32_t)top & 0x7FFFFFu));
}

__device__ __forceinline__ ff ff_from_u64(unsigned long long x) {
  if (x == 0) return {0.f, 0.f};
  const int e = 63 - __clzll((long long)x);
  const unsigned long long rest = e > 23 ? x & ((1ull << (e - 23)) - 1ull) : 0ull;
  return {u64_top24(x), u64_top24(rest)};
}

__device__ __forceinline__ double u64_to_double_rn(unsigned long long x, int scale_exp) {
  if (x == 0) return 0.0;
  int e = 63 - __clzll((long long)x);
  unsigned long long m;
  if (e <= 52) {
    m = x << (52 - e);
  } else {
    const int sh = e - 52;
    unsigned long long q = x >> sh;
    const unsigned long long rem = x & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    if (q >> 53) {
      q >>= 1;
      ++e;
    }
    m = q;
  }
  return __longlong_as_double(
      (long long)(((unsigned long long)(e + 1023 + scale_exp) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return 0.f;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint32_t m = (uint32_t)(b >> 29) & 0x7FFFFFu;
  return __uint_as_float(sign | ((uint32_t)e << 23) | m);
}

// sqrt(x) for float64 x >= 0, within one ulp (correctly rounded but within about
// 2^-69 of a rounding midpoint), with three float64 operations: x = m 4^j with m in
// [1, 4) by the exponent field; sqrt(m) in float-float (about 2^-46), one Newton
// correction y + (m - y^2) / (2y) with the residual from one fused multiply-add
// and the quotient in float32; the result rescaled by 2^j through the exponent
// field. Zero and subnormal x take the float64 square root.
__device__ __forceinline__ double sqrt_nonneg(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e == -1023) return __dsqrt_rn(x);
  const int j = e >> 1;                                // floor(e / 2)
  const double m = __longlong_as_double((long long)(b - ((unsigned long long)(long long)(2 * j) << 52)));
  const ff a = split_nonneg(m);
  const float sh = __fsqrt_rn(a.hi);
  const float h = __fdiv_rn(0.5f, sh);
  const float sl = __fmul_rn(__fadd_rn(__fmaf_rn(-sh, sh, a.hi), a.lo), h);
  const double y = __dadd_rn(f2d_bits(sh), f2d_bits(sl));
  const double r = __fma_rn(-y, y, m);
  const double ym = __dadd_rn(y, f2d_bits(__fmul_rn(d2f_trunc(r), h)));   // sqrt(m) in [1, 2]
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(ym) +
                                          ((unsigned long long)(long long)j << 52)));
}

// e^x for a float-float |x| <= 0.35, from the series definition: the Taylor
// series to degree 12 (remainder below 2^-52), degrees 7..12 in float32 (each
// term below 2^-22 of the result), degrees 0..6 in float-float Horner steps; the
// coefficients 1/m! are stored as float pairs. It fills the table of
// ff_exp_table.
__device__ __forceinline__ ff ff_exp_series(ff x) {
  float p = 0x1.1eed8ep-29f;                      // 1/12!
  p = __fmaf_rn(p, x.hi, 0x1.ae6456p-26f);        // 1/11!
  p = __fmaf_rn(p, x.hi, 0x1.27e4fcp-22f);        // 1/10!
  p = __fmaf_rn(p, x.hi, 0x1.71de3ap-19f);        // 1/9!
  p = __fmaf_rn(p, x.hi, 0x1.a01a02p-16f);        // 1/8!
  p = __fmaf_rn(p, x.hi, 0x1.a01a02p-13f);        // 1/7!
  ff q = {p, 0.f};
  q = ff_add(ff_mul(q, x), ff{0x1.6c16c2p-10f, -0x1.27d27ep-35f});   // 1/6!
  q = ff_add(ff_mul(q, x), ff{0x1.111112p-7f, -0x1.dddddep-32f});    // 1/5!
  q = ff_add(ff_mul(q, x), ff{0x1.555556p-5f, -0x1.555556p-30f});    // 1/4!
  q = ff_add(ff_mul(q, x), ff{0x1.555556p-3f, -0x1.555556p-28f});    // 1/3!
  q = ff_add(ff_mul(q, x), ff{0x1p-1f, 0.f});                        // 1/2!
  q = ff_add(ff_mul(q, x), ff{1.f, 0.f});                            // 1/1!
  q = ff_add(ff_mul(q, x), ff{1.f, 0.f});                            // 1/0!
  return q;
}

// exp(-x y) for float64 x >= 0, y > 0 with x y < 690, as (q.hi + q.lo) 2^-k
// with no float64 operation: the product t = x y is formed exactly as the
// 106-bit product of the two 53-bit mantissas and kept to 64 fractional bits
// (128-bit integers); k = round(t / ln2) from a float estimate; r = t - k ln2
// with ln2 to 64 fractional bits (error below 2^-54 for k < 1024) is a signed
// 64-bit fixed-point number. It is reduced once more, exactly, by j / 32 with j
// = round(32 r) (|j| <= 11): exp(-r) = exp(-j / 32) exp(-r') with |r'| <= 1/64,
// exp(-j / 32) from a table of float-float values (ff_exp_table) and exp(-r')
// from the series to degree 6 (remainder below 2^-54): degrees 4..6 in float32,
// 0..3 in float-float Horner steps. About 1.4e-14 relative, as the degree-12
// series on r alone (a host emulation against quad precision over 2e7
// arguments gives 1.33e-14 and 1.41e-14).
__device__ __forceinline__ ff ff_exp_series6(ff x) {
  float p = 0x1.6c16c2p-10f;                      // 1/6!
  p = __fmaf_rn(p, x.hi, 0x1.111112p-7f);         // 1/5!
  p = __fmaf_rn(p, x.hi, 0x1.555556p-5f);         // 1/4!
  ff q = {p, 0.f};
  q = ff_add(ff_mul(q, x), ff{0x1.555556p-3f, -0x1.555556p-28f});   // 1/3!
  q = ff_add(ff_mul(q, x), ff{0x1p-1f, 0.f});                        // 1/2!
  q = ff_add(ff_mul(q, x), ff{1.f, 0.f});                            // 1/1!
  q = ff_add(ff_mul(q, x), ff{1.f, 0.f});                            // 1/0!
  return q;
}

// exp(-j / 32) for j = -11 .. 11 at tab[j + 11], from the degree-12 series
// (|j / 32| <= 0.35, exact in float). Threads 0 .. 22 of the block fill it;
// the caller synchronises before use.
constexpr int FF_EXP_TABLE = 23;
__device__ __forceinline__ void ff_exp_table(ff* tab) {
  if (threadIdx.x < FF_EXP_TABLE) tab[threadIdx.x] = ff_exp_series(ff{(float)(11 - (int)threadIdx.x) * 0.03125f, 0.f});
}

__device__ __forceinline__ ff ff_exp_neg_prod(double x, double y, int& k_out, const ff* __restrict__ tab) {
  const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
  const unsigned long long by = (unsigned long long)__double_as_longlong(y);
  const int ex = (int)((bx >> 52) & 0x7FF), ey = (int)((by >> 52) & 0x7FF);
  unsigned __int128 T = 0;                                           // t 2^64
  if (ex != 0 && ey != 0) {
    const unsigned long long mx = (bx & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned long long my = (by & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned __int128 P = (unsigned __int128)mx * my;         // t = P 2^(ex + ey - 2150)
    const int sh = ex + ey - 2150 + 64;                              // T = P 2^sh, sh < -30 for t < 2^10
    if (sh >= 0)
      T = P << sh;
    else if (sh > -127)
      T = P >> (-sh);
  }
  const float tf = __fmul_rn(u64_top24((unsigned long long)(T >> 40)), 0x1p-24f);
  const int k = __float2int_rn(__fmul_rn(tf, 0x1.715476p+0f));       // t / ln2
  const unsigned __int128 kl = (unsigned __int128)(unsigned)k * 0xB17217F7D1CF79ABull;   // k ln2 2^64
  const long long r = (long long)(__int128)(T - kl);                 // |r| < 2^63
  long long j = (r + (1ll << 58)) >> 59;                             // round(32 r), |j| <= 11
  j = j < -11 ? -11 : (j > 11 ? 11 : j);                             // (a guard: |r| <= 0.35 here)
  const long long r2 = r - j * (1ll << 59);                          // |r2| <= 2^58: |r'| <= 1/64
  const unsigned long long ar = r2 < 0 ? (unsigned long long)(-r2) : (unsigned long long)r2;
  const ff m = ff_from_u64(ar);
  const float hi = __fmul_rn(m.hi, 0x1p-64f), lo = __fmul_rn(m.lo, 0x1p-64f);   // exact powers of two
  k_out = k;
  const ff e = ff_exp_series6(r2 < 0 ? ff{hi, lo} : ff{-hi, -lo});   // exp(-r')
  return ff_mul(e, tab[j + 11]);                                      // exp(-r), in [0.70, 1.42]
}

// (q.hi + q.lo) 2^-k as float64 for q in [0.5, 2) (q.hi > 0, |q.lo| <= ulp(q.hi)),
// rounded to nearest even, with integer operations only (2^-k in the normal range).
__device__ __forceinline__ double ff_scaled_to_double(ff q, int k) {
  const uint32_t hb = __float_as_uint(q.hi);
  const int eh = (int)((hb >> 23) & 0xFF) - 127;                     // -1 or 0
  long long V = (long long)((hb & 0x7FFFFFu) | 0x800000u) << (eh + 30);   // (q.hi) 2^53
  const uint32_t lb = __float_as_uint(q.lo);
  const int el = (int)((lb >> 23) & 0xFF) - 127;
  if ((lb & 0x7FFFFFFFu) != 0 && el > -127) {
    const long long ml = (long long)((lb & 0x7FFFFFu) | 0x800000u);
    const int s = el + 30;
    const long long L = s >= 0 ? (ml << s) : (s > -64 ? (ml >> (-s)) : 0);
    V += (lb >> 31) ? -L : L;
  }
  int E = -1;
  unsigned long long mant = (unsigned long long)V;                   // leading bit 52 or 53
  if (mant >> 53) {
    const unsigned long long h = mant >> 1;
    mant = h + ((mant & 1ull) & (h & 1ull));                         // ties to even
    E = 0;
  }
  return __longlong_as_double((long long)(((unsigned long long)(E - k + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace cdl
