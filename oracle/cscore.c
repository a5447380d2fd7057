/* Plain C float64 CAD node scores (TEST INFRASTRUCTURE; part of the oracle,
 * shares no code with the CUDA path).
 *
 * Same definition as oracle.caddelag.node_scores (Alg. 4; edge score of
 * Sec. 2; commute times of Eq. 1 through the embedding):
 *   c_t(i, j) = vol_t sum_r (Z_t[i, r] - Z_t[j, r])^2,
 *   F_i = sum_{j != i} |A1_ij - A2_ij| |c_2(i, j) - c_1(i, j)|,
 * with direct differences, r and j in ascending order, one rounding per
 * operation. Rows are independent; OpenMP splits them across threads.
 */
#include <math.h>
#include <stdint.h>

/* rows: node indices (nrows); A1_rows, A2_rows: nrows x n (row t holds row
 * rows[t] of each graph); Z1, Z2: n x k; F: nrows output. */
void cdl_oracle_node_scores(const double* A1_rows, const double* A2_rows, const int64_t* rows, int64_t nrows,
                            int64_t n, const double* Z1, const double* Z2, int32_t k, double vol1, double vol2,
                            double* F) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < nrows; ++t) {
    const int64_t i = rows[t];
    const double* zi1 = Z1 + i * k;
    const double* zi2 = Z2 + i * k;
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dA = fabs(A1_rows[t * n + j] - A2_rows[t * n + j]);
      const double* zj1 = Z1 + j * k;
      const double* zj2 = Z2 + j * k;
      double s1 = 0.0, s2 = 0.0;
      for (int32_t r = 0; r < k; ++r) {
        const double d1 = zi1[r] - zj1[r];
        const double d2 = zi2[r] - zj2[r];
        s1 += d1 * d1;
        s2 += d2 * d2;
      }
      acc += dA * fabs(vol2 * s2 - vol1 * s1);
    }
    F[t] = acc;
  }
}
