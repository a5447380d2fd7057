/* Plain C float64 random projection (TEST INFRASTRUCTURE; part of the
 * oracle, shares no code with the CUDA path).
 *
 * Same definition as oracle.caddelag.project_rows (Alg. 1 / Alg. 3,
 * y = B^T W^{1/2} q edge by edge):
 *   Y[i, r] = k^{-1/2} sum_{j != i} o_ij s_r(min(i,j), max(i,j)) sqrt(A_ij),
 * o_ij = +1 if i < j else -1, s_r = +1 if bit (r mod 32) of word
 * ((r mod 128) / 32) of Philox4x32-10(counter (min, max, r / 128, 0),
 * key (seed low, seed high)) is set, else -1. Philox4x32-10 written from its
 * published definition (Salmon et al., SC'11). Rows are independent; OpenMP
 * splits them across threads; sums run over j in ascending order.
 */
#include <math.h>
#include <stdint.h>

static void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
}

/* sign table: SGN[b][t] = +1 if bit t of byte b is set, else -1 */
static double SGN[256][8];
static void init_sgn(void) {
  for (int b = 0; b < 256; ++b)
    for (int t = 0; t < 8; ++t) SGN[b][t] = ((b >> t) & 1) ? 1.0 : -1.0;
}

/* rows: node indices (nrows); A_rows: nrows x n (row t is row rows[t] of A);
 * Y: nrows x k output. */
void cdl_oracle_project_rows(const double* A_rows, const int64_t* rows, int64_t nrows, int64_t n,
                             int32_t k, uint64_t seed, double* Y) {
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  const int32_t nrb = (k + 127) / 128;
  const double scale = 1.0 / sqrt((double)k);
  init_sgn();
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < nrows; ++t) {
    const int64_t i = rows[t];
    double acc[1024 + 128];
    for (int32_t r = 0; r < 1024 + 128; ++r) acc[r] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const double w = (j > i ? 1.0 : -1.0) * sqrt(A_rows[t * n + j]);
      const uint32_t lo = (uint32_t)(i < j ? i : j), hi = (uint32_t)(i < j ? j : i);
      for (int32_t rb = 0; rb < nrb; ++rb) {
        uint32_t c[4] = {lo, hi, (uint32_t)rb, 0u};
        philox4x32_10(c, k0, k1);
        /* projection row 128 rb + 32 q + 8 m + t <- bit t of byte m of word q;
         * rows >= k accumulate into the spare tail of acc and are discarded */
        for (int32_t q = 0; q < 4; ++q)
          for (int32_t m = 0; m < 4; ++m) {
            const double* sg = SGN[(c[q] >> (8 * m)) & 0xFFu];
            double* a = acc + rb * 128 + 32 * q + 8 * m;
            for (int32_t t = 0; t < 8; ++t) a[t] += sg[t] * w;
          }
      }
    }
    for (int32_t r = 0; r < k; ++r) Y[t * k + r] = acc[r] * scale;
  }
}
