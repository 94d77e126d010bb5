/* CPU oracle for the GDP method on the fractional 2-matching (F2M) LP.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline / reference arm may call this code; the library never does.
 * It is plain, single-threaded, slow and written to be checked by eye against
 * the paper: Section 2 (KKT sign rule (7)), Section 3 (gradient from the b-th and
 * (b+1)-th smallest adjusted values), Section 4 (F2M, Eq. 9 and Eq. 10) and
 * Section 5.1 (per-node and per-edge parallel steps).  It shares no code with
 * the CUDA path.
 *
 * Fixed point: lambda and every reduced cost z are integers in units of
 * 2^-F of a length unit ("F fractional bits").  Costs are TSPLIB EUC_2D
 * lengths, c(u,v) = floor(sqrt(dx^2 + dy^2) + 1/2), integers.
 *
 * Graphs are CSR with both directions stored (row_ptr[n+1], col[nnz]); rows
 * sorted, no self-loops, no duplicates.
 */
#ifndef F2M_ORACLE_H
#define F2M_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_OK = 0,
  OR_INVALID = 1,
  OR_NOT_CONVERGED = 4,
  OR_OVERFLOW = 5,
  OR_PRICING_OVERFLOW = 6,
  OR_INFEASIBLE = 7,
};

/* nearest integer to sqrt(d2): floor(sqrt(d2) + 1/2) evaluated in double */
int64_t or_nint_sqrt(int64_t d2);
void or_nint_sqrt_array(int64_t count, const int64_t* d2, int64_t* out);
/* c(u,v) for points xy[2*u], xy[2*u+1] */
int32_t or_cost(const int32_t* xy, int32_t u, int32_t v);
void or_cost_table(int32_t n, const int32_t* xy, const int32_t* row_ptr,
                   const int32_t* col, int32_t* cost);

/* One Jacobi sweep of GDP (Eq. 9, Eq. 10 with the centring reading):
 * for every node v, from lam_old only,
 *   z_e = c_e*2^F - lam_u - lam_v over the row of v,
 *   z(2) <= z(3) the 2nd and 3rd smallest,
 *   delta_v = trunc((z(2) + z(3)) / 2^shift),  lam_new_v = lam_old_v + delta_v.
 * Also returns bound2 = 4*sum(lam_old) + sum over directed entries of min(0, z)
 * (twice the Lagrangian bound at lam_old, units 2^-F) and changed = #{delta != 0}.
 * b (NULL: every b_v = 2) generalises to the fractional b-matching LP
 * (sum of x over delta(v) = b_v, Section 3's LP3 with b-th and (b+1)-th order
 * statistics): z(b_v) and z(b_v + 1) replace z(2) and z(3), and the bound
 * term 4*lam_v becomes 2*b_v*lam_v.  The same b parameter below has the same
 * meaning.
 * Returns OR_OVERFLOW if some |lam_new| >= 2^29, OR_INVALID on a row of degree
 * below b_v + 1. */
int or_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
             const int32_t* b, const int32_t* lam_old, int32_t F, int32_t shift, int32_t* lam_new,
             int64_t* bound2, int64_t* changed);

/* twice the Lagrangian bound at lam (units 2^-fb) over the CSR edges */
int64_t or_bound2(int32_t n, const int32_t* row_ptr, const int32_t* col,
                  const int32_t* cost, const int32_t* b, const int32_t* lam, int32_t fb);

/* GDP phase: sweeps until a sweep changes nothing or max_iters sweeps ran.
 * lam is updated in place.  iters = sweeps run.  trace_bound2 / trace_changed
 * (may be NULL) receive per-sweep values for the first trace_cap sweeps.
 * Returns OR_OK on a fixed point, OR_NOT_CONVERGED at the cap, OR_OVERFLOW. */
int or_gdp(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
           const int32_t* b, int32_t F, int32_t shift, int64_t max_iters, int32_t* lam, int64_t* iters,
           int64_t* trace_bound2, int64_t* trace_changed, int64_t trace_cap);

/* Sign rule (7): x2_e = 2 if z_e < 0, 1 if z_e == 0, 0 if z_e > 0 (half units).
 * Returns the number of nodes whose row sum of x2 differs from 2 b_v. */
int64_t or_extract(int32_t n, const int32_t* row_ptr, const int32_t* col,
                   const int32_t* cost, const int32_t* b, const int32_t* lam, int32_t fb, uint8_t* x2);

/* Exact finisher: min-cost flow on the bipartite double cover of the CSR graph,
 * warm-started from lam (F bits); plain successive shortest paths over all
 * nodes, sources and Dijkstra ties in key order (L_v: 2v, R_v: 2v + 1).
 * Writes x2 (half units) and lam2 (units 2^-(F+1)).  Returns OR_OK,
 * OR_INFEASIBLE or OR_OVERFLOW. */
int or_finisher(int32_t n, const int32_t* row_ptr, const int32_t* col,
                const int32_t* cost, const int32_t* b, const int32_t* lam, int32_t F, uint8_t* x2,
                int32_t* lam2, int64_t* augmentations);

/* Pricing: every pair u < v that is not an edge of the CSR and has
 * c(u,v)*2^fb < lam_u + lam_v.  Writes up to cap pairs (u, v) in ascending
 * (u, v) order into pairs[2*i], pairs[2*i+1]; returns the total count. */
int64_t or_pricing(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
                   const int32_t* lam, int32_t fb, int32_t* pairs, int64_t cap);

/* Pricing restricted to rows u in [u_begin, u_end) (a bounded sample of the scan). */
int64_t or_pricing_rows(int32_t n, const int32_t* xy, const int32_t* row_ptr,
                        const int32_t* col, const int32_t* lam, int32_t fb,
                        int32_t u_begin, int32_t u_end, int32_t* pairs, int64_t cap);

/* Union of a CSR with undirected pairs (both directions), rows sorted.
 * out_row_ptr has n+1 entries; out_col needs nnz + 2*npairs entries.
 * Returns the new nnz. */
int64_t or_merge(int32_t n, const int32_t* row_ptr, const int32_t* col, int64_t npairs,
                 const int32_t* pairs, int32_t* out_row_ptr, int32_t* out_col);

/* Full solve, Section 4-5 with pricing and finisher (see f2m_oracle.c). */
/* Colour classes and the class-by-class (Gauss-Seidel) variant of the sweep.
 * or_splitmix64: first output of SplitMix64 seeded with `seed`.
 * or_color_greedy: greedy colouring (smallest colour unused by coloured
 *   neighbours) in priority order: larger degree, then larger
 *   or_splitmix64(v), then smaller v.  Returns the number of colours.
 * or_gs_sweep: one sweep updating lam IN PLACE class 0, 1, ..., ncolors-1, each
 *   node of the class from the current lambda (Eq. 9; Eq. 10 or its b_v form).
 *   bound2 = the bound at the input lambda (as or_bound2); changed = #{delta != 0}.
 *   A node whose new value would reach |lambda| >= 2^29 keeps its value, the
 *   sweep completes and OR_OVERFLOW is returned; OR_INVALID on a short row.
 * or_gdp_gs: sweeps until one changes nothing or max_iters (as or_gdp). */
uint64_t or_splitmix64(uint64_t seed);
int32_t or_color_greedy(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* color);
int or_gs_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                const int32_t* b, const int32_t* color, int32_t ncolors, int32_t* lam, int32_t F,
                int32_t shift, int64_t* bound2, int64_t* changed);
int or_gdp_gs(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
              const int32_t* b, const int32_t* color, int32_t ncolors, int32_t F, int32_t shift,
              int64_t max_iters, int32_t* lam, int64_t* iters, int64_t* trace_bound2,
              int64_t* trace_changed, int64_t trace_cap);

typedef struct {
  int32_t frac_bits;        /* F */
  int32_t damping_shift;    /* shift in delta = trunc((z2+z3)/2^shift) */
  int64_t max_iters;        /* per GDP phase */
  int32_t max_pricing_rounds;
  int32_t pricing;          /* 0 off, 1 full */
  int32_t finisher;         /* 0 off, 1 on */
  int32_t update;           /* OR_UPDATE_JACOBI or OR_UPDATE_CLASSES */
} or_params;

#define OR_UPDATE_JACOBI 0   /* Section 5.1: all nodes from one lambda (or_gdp) */
#define OR_UPDATE_CLASSES 1  /* colour class by colour class (or_gdp_gs) */

typedef struct {
  int64_t iterations;       /* total sweeps over all phases */
  int64_t phases;           /* GDP phases run */
  int64_t pricing_rounds;   /* pricing scans run */
  int64_t edges_added;      /* undirected edges added by pricing */
  int64_t finisher_calls;
  int64_t augmentations;
  int64_t bound2;           /* 2*LB in units 2^-frac_bits */
  int32_t frac_bits;        /* F, or F+1 after the finisher */
  int32_t certified;        /* 0 none, 1 optimal on the candidate graph, 2 globally */
  int32_t status;
} or_info;

typedef struct or_result or_result;

/* lam0: initial lambda (F bits) or NULL for zero.  trace arrays as in or_gdp
 * (one entry per sweep, all phases concatenated). */
or_result* or_solve(int32_t n, const int32_t* xy, const int32_t* row_ptr,
                    const int32_t* col, const int32_t* b, const int32_t* lam0, const or_params* p,
                    or_info* info, int64_t* trace_bound2, int64_t* trace_changed,
                    int64_t trace_cap);
int64_t or_result_nnz(const or_result* r);
/* row_ptr[n+1], col[nnz], x2[nnz], lam[n] (units 2^-info.frac_bits) */
void or_result_copy(const or_result* r, int32_t* row_ptr, int32_t* col, uint8_t* x2,
                    int32_t* lam);
void or_result_free(or_result* r);

/* k nearest neighbours of every point (the candidate graph of Section 5.3 and
 * the warm-start features): the k other points with the smallest exact squared
 * distance dx^2 + dy^2 (int64), ties broken by smaller index; copies of the
 * point at distance 0 count, the point itself does not.  Brute force over all
 * pairs.  nbr[i*k + j] and d2[i*k + j], j = 0..k-1, in that order.  Needs
 * n > k. */
void or_knn(int32_t n, const int32_t* xy, int32_t k, int32_t* nbr, int64_t* d2);

/* Certificate (independent of the solver): returns 0 when all checks pass,
 * else the number of the first failed check (see certify.c). */
int or_certify(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
               const int32_t* b, const uint8_t* x2, const int32_t* lam, int32_t fb, int64_t bound2,
               int32_t full_scan);


/* ---- subtour-elimination cuts (subtour.c) ----------------------------------
 * GDP on F2M plus cuts x(delta(S)) >= 2 of a layered family (see subtour.c):
 * comp [L][n] labels (-1: no cut of the layer), ncuts [L], mu [sum ncuts]
 * (units 2^-F, >= 0). */
int64_t or_cut_z(int32_t n, const int32_t* xy, int32_t L, const int32_t* comp, const int32_t* ncuts,
                 const int32_t* lam, const int32_t* mu, int32_t fb, int32_t u, int32_t v);
int64_t or_cut_bound2(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                      int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam,
                      const int32_t* mu, int32_t fb);
int or_cut_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                 int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam_old,
                 const int32_t* mu_old, int32_t F, int32_t shift, int32_t* lam_new, int32_t* mu_new,
                 int64_t* bound2, int64_t* changed);
int or_cut_gdp(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost, int32_t L,
               const int32_t* comp, const int32_t* ncuts, int32_t F, int32_t shift, int64_t max_iters,
               int32_t* lam, int32_t* mu, int64_t* iters, int64_t* trace_bound2, int64_t* trace_changed,
               int64_t trace_cap);
int64_t or_cut_extract(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                       int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam,
                       const int32_t* mu, int32_t fb, uint8_t* x2);
/* components of the support of x2 as one cut layer: writes comp [n], returns
 * the number of cuts */
int32_t or_separate(int32_t n, const int32_t* row_ptr, const int32_t* col, const uint8_t* x2,
                    int32_t* comp);
int64_t or_cut_pricing(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
                       int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam,
                       const int32_t* mu, int32_t fb, int32_t* pairs, int64_t cap);

typedef struct {
  int64_t iterations, phases, pricing_rounds, edges_added, cuts;
  int64_t bound2_f2m;   /* 2*LB after stage 0 (no cuts), units 2^-F */
  int64_t bound2;       /* 2*LB at the end */
  int32_t rounds, layers, frac_bits, certified, status;
} or_subtour_info;
typedef struct or_subtour or_subtour;
/* stages of GDP with pricing and cut layers between them (see subtour.c);
 * lam0 NULL: zero */
or_subtour* or_solve_subtour(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
                             const int32_t* lam0, int32_t F, int32_t shift, int64_t max_iters,
                             int32_t pricing, int32_t max_pricing_rounds, int32_t rounds,
                             or_subtour_info* info);
int64_t or_subtour_nnz(const or_subtour* r);
int64_t or_subtour_cuts(const or_subtour* r);
int32_t or_subtour_layers(const or_subtour* r);
void or_subtour_copy(const or_subtour* r, int32_t* row_ptr, int32_t* col, uint8_t* x2, int32_t* lam,
                     int32_t* mu, int32_t* comp, int32_t* ncuts);
void or_subtour_free(or_subtour* r);

#ifdef __cplusplus
}
#endif
#endif
