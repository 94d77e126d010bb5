/* Optimality certificate for an F2M solution -- TEST INFRASTRUCTURE ONLY.
 *
 * Written separately from the oracle solver (it computes costs with integer
 * arithmetic only and shares no helper with f2m_oracle.c), so a solver bug is
 * not repeated here.  Given points, a CSR graph, x in half units (x2) and a
 * dual lambda in units 2^-fb, it checks LP optimality over the COMPLETE graph
 * of the points (the F2M LP of Section 4):
 *   1  every x2 is 0, 1 or 2;
 *   2  x2 agrees on both directions of an edge;
 *   3  every node has row sum 2 b_v, i.e. sum of x over delta(v) = b_v (b_v = 2
 *      for the fractional 2-matching; other b_v for a fractional b-matching);
 *   4  complementary slackness with z = c*2^fb - lam_u - lam_v (rule (7)):
 *      x = 1 -> z <= 0, x = 1/2 -> z == 0, x = 0 -> z >= 0;
 *   5  bound2 = 2*sum(b_v lam_v) + sum over directed entries of min(0, z);
 *   6  primal cost equals the dual bound: sum_dir x2 * c * 2^fb == 2 * bound2;
 *   7  (full_scan) no pair outside the graph has z < 0, so the duals
 *      mu_e = max(0, -z_e) with lambda are feasible for the complete graph.
 * Checks 1-6 make (x, lambda) optimal on the graph; with 7 the optimum is
 * that of the complete graph.  Returns 0 or the number of the failed check.
 */
#include <stdint.h>
#include <stdlib.h>

/* floor(sqrt(a)) for a >= 0, bit-by-bit (no floating point) */
static int64_t cert_isqrt(int64_t a) {
  int64_t r = 0, bit = (int64_t)1 << 62;
  while (bit > a) bit >>= 2;
  while (bit) {
    if (a >= r + bit) { a -= r + bit; r = (r >> 1) + bit; }
    else r >>= 1;
    bit >>= 2;
  }
  return r;
}

/* nearest integer to sqrt(d2) = floor((isqrt(4*d2) + 1) / 2) */
static int64_t cert_len(const int32_t* xy, int32_t u, int32_t v) {
  int64_t dx = (int64_t)xy[2 * (int64_t)u] - xy[2 * (int64_t)v];
  int64_t dy = (int64_t)xy[2 * (int64_t)u + 1] - xy[2 * (int64_t)v + 1];
  return (cert_isqrt(4 * (dx * dx + dy * dy)) + 1) >> 1;
}

int or_certify(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
               const int32_t* b, const uint8_t* x2, const int32_t* lam, int32_t fb, int64_t bound2,
               int32_t full_scan) {
  int64_t b2 = 0, primal = 0;
  for (int32_t u = 0; u < n; ++u) {
    int32_t s = 0;
    const int32_t bu = b ? b[u] : 2;
    b2 += 2 * (int64_t)bu * lam[u];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      if (x2[e] > 2) return 1;
      int32_t back = -1;
      for (int32_t f = row_ptr[v]; f < row_ptr[v + 1]; ++f)
        if (col[f] == u) back = f;
      if (back < 0 || x2[back] != x2[e]) return 2;
      s += x2[e];
      int64_t c = cert_len(xy, u, v);
      int64_t z = c * ((int64_t)1 << fb) - lam[u] - lam[v];
      if (x2[e] == 2 && z > 0) return 4;
      if (x2[e] == 1 && z != 0) return 4;
      if (x2[e] == 0 && z < 0) return 4;
      if (z < 0) b2 += z;
      primal += (int64_t)x2[e] * c * ((int64_t)1 << fb);
    }
    if (s != 2 * bu) return 3;
  }
  if (b2 != bound2) return 5;
  if (primal != 2 * bound2) return 6;
  if (full_scan) {
    char* in = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int32_t u = 0; u < n; ++u) {
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) in[col[e]] = 1;
      for (int32_t v = u + 1; v < n; ++v) {
        if (in[v]) continue;
        int64_t S = (int64_t)lam[u] + lam[v];
        if (S <= 0) continue; /* c >= 0, so z >= 0 */
        /* z < 0  <=>  c < S / 2^fb  <=>  c <= m, m = ceil(S / 2^fb) - 1
         *        <=>  sqrt(d2) < m + 1/2  <=>  4*d2 < (2m + 1)^2 */
        int64_t m = ((S + ((int64_t)1 << fb) - 1) >> fb) - 1;
        int64_t dx = (int64_t)xy[2 * (int64_t)u] - xy[2 * (int64_t)v];
        int64_t dy = (int64_t)xy[2 * (int64_t)u + 1] - xy[2 * (int64_t)v + 1];
        if (4 * (dx * dx + dy * dy) < (2 * m + 1) * (2 * m + 1)) { free(in); return 7; }
      }
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) in[col[e]] = 0;
    }
    free(in);
  }
  return 0;
}
