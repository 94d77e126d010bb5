/* CPU oracle for GDP on the fractional 2-matching LP -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline / reference arm
 * load this file's library.  The product path (the CUDA library) never does and
 * shares no code with it.  Plain, single-threaded, written for checking by eye.
 *
 * Paper passages followed (arXiv 2011.08170):
 *   Section 2, rule (7): sign of the modified objective v gives x in {1, frac, 0}.
 *   Section 3: for a constraint with binary coefficients and integral right side
 *     b, the gradient is taken from the b-th and (b+1)-th smallest values of v
 *     over its support.
 *   Section 4, Eq. (9): adjusted edge length v^e = c^e - lambda_u - lambda_v.
 *   Section 4, Eq. (10): gradient of lambda_v from the 2nd and 3rd shortest
 *     adjusted edges at v (b = 2).
 *   Section 4: the F2M optimum is {0, 1/2, 1} valued (Edmonds).
 *   Section 5.1: gradient per node and update per edge, in parallel (Jacobi).
 *   Section 5.3 / Tables 1a, 2: top-N nearest-neighbour candidate graph.
 *
 * Readings where the paper is silent or garbled (each is a parameter or a
 * stated choice):
 *   - Eq. (10) prints 0.5*(v2 - v3), which is never positive for sorted values.
 *     The step used is the one that centres the 2nd and 3rd adjusted lengths on
 *     zero: a full centring step is (z2 + z3)/2, after which they become
 *     -/+ (z3 - z2)/2, the magnitude Eq. (10) prints.  Because Jacobi moves both
 *     ends of an edge at once, the default takes half of it, (z2 + z3)/4
 *     (damping_shift = 2); damping_shift = 1 is the full step.
 *   - Precision: lambda in fixed point, F = 8 fractional bits, int32; the
 *     quotient is truncated toward zero (C division), which leaves a symmetric
 *     dead zone so an exact fixed point exists.
 *   - Stop: a sweep that changes no lambda, or max_iters sweeps; either way the
 *     solve goes on from the lambda reached (pricing, rule (7), finisher).
 *   - Degenerate stops (Section 3, last paragraph: the constraint values are not
 *     controlled) are resolved by an exact min-cost-flow finisher.
 *   - Candidate graphs can miss optimal edges (Section 5.3); a pricing scan over
 *     all pairs adds every edge with negative reduced cost, then GDP resumes.
 */
#include "f2m_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_LAM_LIMIT (1LL << 29)

/* ---- costs: TSPLIB EUC_2D nearest-integer Euclidean length ---------------- */

int64_t or_nint_sqrt(int64_t d2) { return (int64_t)floor(sqrt((double)d2) + 0.5); }

void or_nint_sqrt_array(int64_t count, const int64_t* d2, int64_t* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = or_nint_sqrt(d2[i]);
}

int32_t or_cost(const int32_t* xy, int32_t u, int32_t v) {
  int64_t dx = (int64_t)xy[2 * (int64_t)u] - xy[2 * (int64_t)v];
  int64_t dy = (int64_t)xy[2 * (int64_t)u + 1] - xy[2 * (int64_t)v + 1];
  return (int32_t)or_nint_sqrt(dx * dx + dy * dy);
}

void or_cost_table(int32_t n, const int32_t* xy, const int32_t* row_ptr,
                   const int32_t* col, int32_t* cost) {
  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) cost[e] = or_cost(xy, u, col[e]);
}

/* ---- one GDP sweep: Eq. (9) per entry, Eq. (10) per node ------------------ */

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

int or_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
             const int32_t* b, const int32_t* lam_old, int32_t F, int32_t shift, int32_t* lam_new,
             int64_t* bound2, int64_t* changed) {
  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
  int64_t* z = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxdeg > 0 ? maxdeg : 1));
  int64_t b2 = 0, ch = 0;
  int status = OR_OK;
  for (int32_t v = 0; v < n; ++v) {
    int32_t deg = row_ptr[v + 1] - row_ptr[v];
    int32_t bv = b ? b[v] : 2;
    if (bv < 1 || deg < bv + 1) { status = OR_INVALID; break; }
    for (int32_t j = 0; j < deg; ++j) {
      int32_t e = row_ptr[v] + j;
      /* Eq. (9): adjusted length of edge (v, col[e]) */
      z[j] = ((int64_t)cost[e] << F) - lam_old[v] - lam_old[col[e]];
      if (z[j] < 0) b2 += z[j];
    }
    b2 += 2 * (int64_t)bv * lam_old[v];
    /* Eq. (10): 2nd and 3rd shortest adjusted edges at v; for a degree
     * requirement b_v (Section 3), the b_v-th and (b_v+1)-th */
    qsort(z, (size_t)deg, sizeof(int64_t), cmp_i64);
    int64_t delta = (z[bv - 1] + z[bv]) / ((int64_t)1 << shift); /* C division: toward zero */
    int64_t nl = (int64_t)lam_old[v] + delta;
    if (nl >= OR_LAM_LIMIT || nl <= -OR_LAM_LIMIT) status = OR_OVERFLOW;
    lam_new[v] = (int32_t)nl;
    if (delta != 0) ++ch;
  }
  free(z);
  *bound2 = b2;
  *changed = ch;
  return status;
}

int64_t or_bound2(int32_t n, const int32_t* row_ptr, const int32_t* col,
                  const int32_t* cost, const int32_t* b, const int32_t* lam, int32_t fb) {
  int64_t b2 = 0;
  for (int32_t v = 0; v < n; ++v) {
    b2 += 2 * (int64_t)(b ? b[v] : 2) * lam[v];
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int64_t z = ((int64_t)cost[e] << fb) - lam[v] - lam[col[e]];
      if (z < 0) b2 += z;
    }
  }
  return b2;
}

int or_gdp(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
           const int32_t* b, int32_t F, int32_t shift, int64_t max_iters, int32_t* lam, int64_t* iters,
           int64_t* trace_bound2, int64_t* trace_changed, int64_t trace_cap) {
  int32_t* nxt = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int status = OR_NOT_CONVERGED;
  int64_t it = 0;
  while (it < max_iters) {
    int64_t b2, ch;
    int st = or_sweep(n, row_ptr, col, cost, b, lam, F, shift, nxt, &b2, &ch);
    if (it < trace_cap) {
      if (trace_bound2) trace_bound2[it] = b2;
      if (trace_changed) trace_changed[it] = ch;
    }
    ++it;
    if (st != OR_OK) { status = st; break; }
    memcpy(lam, nxt, sizeof(int32_t) * (size_t)n);
    if (ch == 0) { status = OR_OK; break; }
  }
  free(nxt);
  *iters = it;
  return status;
}

/* ---- colour classes and the class-by-class (Gauss-Seidel) sweep -----------
 * Section 5.1 computes every node's gradient in parallel from one lambda
 * (Jacobi, or_sweep).  The variant below updates one colour class at a time, a
 * class being an independent set of the graph: nodes of a class share no edge,
 * so their updates do not interact, and each node reads the current lambda of
 * its neighbours.  With the full step (shift = 1) each class update maximises
 * the Lagrangian over that class's duals with the others fixed, so the bound
 * never decreases from sweep to sweep.  The paper does not describe this
 * variant; it is a stated extension.
 *
 * Colouring: greedy, each node taking the smallest colour not held by an
 * already-coloured neighbour, nodes taken in priority order: larger degree
 * first, then larger h(v), then smaller id, where h(v) is the first output of
 * SplitMix64 (Steele, Lea and Flood 2014) seeded with v. */

uint64_t or_splitmix64(uint64_t seed) {
  uint64_t z = seed + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static const int32_t* g_color_rp; /* qsort context for cmp_priority */

static int cmp_priority(const void* a, const void* b) {
  int32_t u = *(const int32_t*)a, v = *(const int32_t*)b;
  int32_t du = g_color_rp[u + 1] - g_color_rp[u], dv = g_color_rp[v + 1] - g_color_rp[v];
  if (du != dv) return du > dv ? -1 : 1;
  uint64_t hu = or_splitmix64((uint64_t)u), hv = or_splitmix64((uint64_t)v);
  if (hu != hv) return hu > hv ? -1 : 1;
  return (u > v) - (u < v);
}

int32_t or_color_greedy(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* color) {
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v) {
    order[v] = v;
    color[v] = -1;
    if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
  }
  g_color_rp = row_ptr;
  qsort(order, (size_t)n, sizeof(int32_t), cmp_priority);
  uint8_t* used = (uint8_t*)calloc((size_t)maxdeg + 2, 1);
  int32_t ncolors = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t v = order[i];
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int32_t c = color[col[e]];
      if (c >= 0 && c <= maxdeg) used[c] = 1;
    }
    int32_t c = 0;
    while (used[c]) ++c;
    color[v] = c;
    if (c + 1 > ncolors) ncolors = c + 1;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int32_t cc = color[col[e]];
      if (cc >= 0 && cc <= maxdeg) used[cc] = 0;
    }
  }
  free(used);
  free(order);
  return ncolors;
}

int or_gs_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                const int32_t* b, const int32_t* color, int32_t ncolors, int32_t* lam, int32_t F,
                int32_t shift, int64_t* bound2, int64_t* changed) {
  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
  int64_t* z = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxdeg > 0 ? maxdeg : 1));
  *bound2 = or_bound2(n, row_ptr, col, cost, b, lam, F); /* at the sweep's input */
  int64_t ch = 0;
  int status = OR_OK;
  for (int32_t c = 0; c < ncolors && status != OR_INVALID; ++c) {
    for (int32_t v = 0; v < n; ++v) {
      if (color[v] != c) continue;
      int32_t deg = row_ptr[v + 1] - row_ptr[v];
      int32_t bv = b ? b[v] : 2;
      if (bv < 1 || deg < bv + 1) { status = OR_INVALID; break; }
      for (int32_t j = 0; j < deg; ++j) {
        int32_t e = row_ptr[v] + j;
        z[j] = ((int64_t)cost[e] << F) - lam[v] - lam[col[e]]; /* Eq. (9), current lambda */
      }
      qsort(z, (size_t)deg, sizeof(int64_t), cmp_i64);
      int64_t delta = (z[bv - 1] + z[bv]) / ((int64_t)1 << shift); /* Eq. (10) / Section 3 */
      int64_t nl = (int64_t)lam[v] + delta;
      if (delta != 0) ++ch;
      if (nl >= OR_LAM_LIMIT || nl <= -OR_LAM_LIMIT) { status = OR_OVERFLOW; continue; } /* keeps its value */
      lam[v] = (int32_t)nl;
    }
  }
  free(z);
  *changed = ch;
  return status;
}

int or_gdp_gs(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
              const int32_t* b, const int32_t* color, int32_t ncolors, int32_t F, int32_t shift,
              int64_t max_iters, int32_t* lam, int64_t* iters, int64_t* trace_bound2,
              int64_t* trace_changed, int64_t trace_cap) {
  int status = OR_NOT_CONVERGED;
  int64_t it = 0;
  while (it < max_iters) {
    int64_t b2, ch;
    int st = or_gs_sweep(n, row_ptr, col, cost, b, color, ncolors, lam, F, shift, &b2, &ch);
    if (it < trace_cap) {
      if (trace_bound2) trace_bound2[it] = b2;
      if (trace_changed) trace_changed[it] = ch;
    }
    ++it;
    if (st != OR_OK) { status = st; break; }
    if (ch == 0) { status = OR_OK; break; }
  }
  *iters = it;
  return status;
}

/* ---- rule (7): primal from the signs of the adjusted lengths -------------- */

int64_t or_extract(int32_t n, const int32_t* row_ptr, const int32_t* col,
                   const int32_t* cost, const int32_t* b, const int32_t* lam, int32_t fb, uint8_t* x2) {
  int64_t bad = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t s = 0;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int64_t z = ((int64_t)cost[e] << fb) - lam[v] - lam[col[e]];
      x2[e] = (uint8_t)(z < 0 ? 2 : (z == 0 ? 1 : 0));
      s += x2[e];
    }
    if (s != 2 * (b ? b[v] : 2)) ++bad;
  }
  return bad;
}

/* ---- exact finisher: min-cost flow on the bipartite double cover ----------
 * Section 3 (last paragraph) leaves the repair of degenerate stops to the
 * problem at hand.  For F2M it is exact: the fractional 2-matching LP on a
 * graph is half of the transportation problem on its bipartite double cover.
 * Node ids: left copy L_v = v, right copy R_v = n + v.  Entry e = (u -> v) is
 * the arc L_u -> R_v, capacity 1, cost C_e = c_e * 2^F.  Every L_v has supply b_v
 * (2 for the fractional 2-matching), every R_v demand b_v.
 * x_uv = (y(L_u R_v) + y(L_v R_u)) / 2 is an optimal F2M
 * point and lambda_v = (pi(L_v) - pi(R_v)) / 2 an optimal dual (units 2^-F),
 * i.e. pi(L_v) - pi(R_v) in units 2^-(F+1).
 * Reduced cost of a residual arc i -> j: C(i, j) - pi(i) + pi(j).
 * Warm start: pi(L_v) = lam_v, pi(R_v) = -lam_v (reduced cost of an arc = z_e),
 * arcs with z_e < 0 saturated, so every residual reduced cost is >= 0.
 * Successive shortest paths (the textbook primal-dual method), one unit at a
 * time: take the node with positive excess and the smallest key, run Dijkstra
 * on the reduced costs from it (heap order: distance, then key) to the first
 * settled node t with negative excess, push one unit along the path, and raise
 * pi(i) by d(t) - d(i) on every node i settled before t.  Key of a node: 2v for
 * L_v and 2v + 1 for R_v.  (The paper gives no finisher; the key order is a
 * stated choice that makes the result deterministic.)  A source from which no
 * deficit node is reachable means the graph has no fractional 2-matching. */

typedef struct { int64_t d; int32_t key; int32_t v; } or_hitem;

static int or_hless(or_hitem a, or_hitem b) { return a.d < b.d || (a.d == b.d && a.key < b.key); }

static void or_hpush(or_hitem* h, int64_t* sz, or_hitem it) {
  int64_t i = (*sz)++;
  h[i] = it;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!or_hless(h[i], h[p])) break;
    or_hitem t = h[i]; h[i] = h[p]; h[p] = t; i = p;
  }
}

static or_hitem or_hpop(or_hitem* h, int64_t* sz) {
  or_hitem top = h[0];
  h[0] = h[--(*sz)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *sz && or_hless(h[l], h[m])) m = l;
    if (r < *sz && or_hless(h[r], h[m])) m = r;
    if (m == i) break;
    or_hitem t = h[i]; h[i] = h[m]; h[m] = t; i = m;
  }
  return top;
}

static int32_t or_find(const int32_t* row_ptr, const int32_t* col, int32_t u, int32_t v) {
  int32_t lo = row_ptr[u], hi = row_ptr[u + 1] - 1;
  while (lo <= hi) {
    int32_t mid = lo + (hi - lo) / 2;
    if (col[mid] == v) return mid;
    if (col[mid] < v) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static int32_t or_key(int32_t n, int32_t i) { return i < n ? 2 * i : 2 * (i - n) + 1; }

int or_finisher(int32_t n, const int32_t* row_ptr, const int32_t* col,
                const int32_t* cost, const int32_t* b, const int32_t* lam, int32_t F, uint8_t* x2,
                int32_t* lam2, int64_t* augmentations) {
  int64_t nnz = row_ptr[n];
  int32_t N = 2 * n;
  size_t ne = (size_t)(nnz > 0 ? nnz : 1);
  int32_t* rev = (int32_t*)malloc(sizeof(int32_t) * ne);  /* entry (v -> u) of entry (u -> v) */
  int32_t* own = (int32_t*)malloc(sizeof(int32_t) * ne);  /* row of each entry */
  uint8_t* y = (uint8_t*)calloc(ne, 1);                   /* flow on arc L_u -> R_v */
  int64_t* pi = (int64_t*)calloc((size_t)N, sizeof(int64_t));
  int64_t* ex = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  int64_t* dist = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  int32_t* par = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);   /* entry used to reach */
  int64_t* seen = (int64_t*)calloc((size_t)N, sizeof(int64_t));   /* stamp: reached */
  int64_t* done = (int64_t*)calloc((size_t)N, sizeof(int64_t));   /* stamp: settled */
  int32_t* settled = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  or_hitem* heap = (or_hitem*)malloc(sizeof(or_hitem) * (size_t)(nnz + N + 1));
  int status = OR_OK;
  int64_t aug = 0;

  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      rev[e] = or_find(row_ptr, col, col[e], u);
      own[e] = u;
    }
  for (int32_t v = 0; v < n; ++v) { pi[v] = lam[v]; pi[n + v] = -(int64_t)lam[v]; }
  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int64_t z = ((int64_t)cost[e] << F) - lam[u] - lam[col[e]];
      y[e] = (uint8_t)(z < 0);
    }
  for (int32_t u = 0; u < n; ++u) {
    int64_t out = 0, in = 0;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) { out += y[e]; in += y[rev[e]]; }
    const int64_t bu = b ? b[u] : 2;
    ex[u] = bu - out;      /* L_u: supply b_u minus outflow */
    ex[n + u] = in - bu;   /* R_u: inflow minus demand b_u */
  }

  /* Excess of a source only falls and a deficit node only fills, so taking the
   * keys once in ascending order is taking the smallest key with excess. */
  int64_t stamp = 0;
  for (int32_t k = 0; k < N && status == OR_OK; ++k) {
    const int32_t src = (k & 1) ? n + k / 2 : k / 2; /* the node with key k */
    while (ex[src] > 0) {
      ++stamp;
      int64_t hs = 0, ns = 0;
      int32_t t = -1;
      dist[src] = 0; seen[src] = stamp; par[src] = -1;
      or_hpush(heap, &hs, (or_hitem){0, or_key(n, src), src});
      while (hs > 0) {
        or_hitem it = or_hpop(heap, &hs);
        int32_t i = it.v;
        if (done[i] == stamp || it.d != dist[i]) continue;
        done[i] = stamp;
        if (ex[i] < 0) { t = i; break; }
        settled[ns++] = i;
        if (i < n) { /* L_i: forward arcs with no flow */
          for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (y[e]) continue;
            int32_t j = n + col[e];
            int64_t nd = dist[i] + ((int64_t)cost[e] << F) - pi[i] + pi[j];
            if (done[j] != stamp && (seen[j] != stamp || nd < dist[j])) {
              seen[j] = stamp; dist[j] = nd; par[j] = e;
              or_hpush(heap, &hs, (or_hitem){nd, or_key(n, j), j});
            }
          }
        } else { /* R_v: reverse arcs of saturated entries (u -> v) */
          int32_t v = i - n;
          for (int32_t f = row_ptr[v]; f < row_ptr[v + 1]; ++f) {
            int32_t e = rev[f]; /* entry (col[f] -> v) */
            if (!y[e]) continue;
            int32_t j = col[f];
            int64_t nd = dist[i] - ((int64_t)cost[e] << F) - pi[i] + pi[j];
            if (done[j] != stamp && (seen[j] != stamp || nd < dist[j])) {
              seen[j] = stamp; dist[j] = nd; par[j] = e;
              or_hpush(heap, &hs, (or_hitem){nd, or_key(n, j), j});
            }
          }
        }
      }
      if (t < 0) { status = OR_INFEASIBLE; break; }
      /* push one unit along the path, walking back from t to src */
      for (int32_t j = t; j != src;) {
        int32_t e = par[j];
        if (j >= n) { y[e] = 1; j = own[e]; }      /* reached R_v by L_u -> R_v, e = (u -> v) */
        else { y[e] = 0; j = n + col[e]; }         /* reached L_u by R_v -> L_u, e = (u -> v) */
      }
      ex[src] -= 1;
      ex[t] += 1;
      ++aug;
      int64_t dt = dist[t];
      for (int64_t q = 0; q < ns; ++q) {
        int32_t i = settled[q];
        pi[i] += dt - dist[i];
      }
    }
  }

  if (status == OR_OK) {
    for (int32_t u = 0; u < n; ++u)
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) x2[e] = (uint8_t)(y[e] + y[rev[e]]);
    for (int32_t v = 0; v < n; ++v) {
      int64_t l2 = pi[v] - pi[n + v];
      if (l2 >= 2 * OR_LAM_LIMIT || l2 <= -2 * OR_LAM_LIMIT) status = OR_OVERFLOW;
      lam2[v] = (int32_t)l2;
    }
  }
  *augmentations = aug;
  free(rev); free(own); free(y); free(pi); free(ex); free(dist); free(par);
  free(seen); free(done); free(settled); free(heap);
  return status;
}

/* ---- pricing: every non-candidate pair with negative adjusted length ------
 * Plain double loop over u < v with the cost recomputed from the points. */

int64_t or_pricing_rows(int32_t n, const int32_t* xy, const int32_t* row_ptr,
                        const int32_t* col, const int32_t* lam, int32_t fb,
                        int32_t u_begin, int32_t u_end, int32_t* pairs, int64_t cap) {
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) mark[v] = -1;
  int64_t count = 0;
  for (int32_t u = u_begin; u < u_end; ++u) {
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) mark[col[e]] = u;
    for (int32_t v = u + 1; v < n; ++v) {
      if (mark[v] == u) continue; /* already a candidate edge */
      int64_t z = ((int64_t)or_cost(xy, u, v) << fb) - lam[u] - lam[v];
      if (z < 0) {
        if (count < cap) { pairs[2 * count] = u; pairs[2 * count + 1] = v; }
        ++count;
      }
    }
  }
  free(mark);
  return count;
}

int64_t or_pricing(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
                   const int32_t* lam, int32_t fb, int32_t* pairs, int64_t cap) {
  return or_pricing_rows(n, xy, row_ptr, col, lam, fb, 0, n, pairs, cap);
}

/* ---- union of the CSR with new undirected pairs --------------------------- */

static int cmp_pair(const void* a, const void* b) {
  const int32_t* x = (const int32_t*)a;
  const int32_t* y = (const int32_t*)b;
  if (x[0] != y[0]) return (x[0] > y[0]) - (x[0] < y[0]);
  return (x[1] > y[1]) - (x[1] < y[1]);
}

int64_t or_merge(int32_t n, const int32_t* row_ptr, const int32_t* col, int64_t npairs,
                 const int32_t* pairs, int32_t* out_row_ptr, int32_t* out_col) {
  /* both directions of every new pair, sorted by (row, column) */
  int32_t* dir = (int32_t*)malloc(sizeof(int32_t) * (size_t)(4 * npairs + 2));
  for (int64_t i = 0; i < npairs; ++i) {
    dir[4 * i] = pairs[2 * i];     dir[4 * i + 1] = pairs[2 * i + 1];
    dir[4 * i + 2] = pairs[2 * i + 1]; dir[4 * i + 3] = pairs[2 * i];
  }
  qsort(dir, (size_t)(2 * npairs), 2 * sizeof(int32_t), cmp_pair);
  int64_t k = 0, out = 0;
  out_row_ptr[0] = 0;
  for (int32_t u = 0; u < n; ++u) {
    int32_t e = row_ptr[u];
    for (;;) {
      int has_old = e < row_ptr[u + 1];
      int has_new = k < 2 * npairs && dir[2 * k] == u;
      if (!has_old && !has_new) break;
      int32_t c;
      if (has_old && (!has_new || col[e] <= dir[2 * k + 1])) {
        c = col[e];
        if (has_new && dir[2 * k + 1] == c) ++k; /* already present */
        ++e;
      } else {
        c = dir[2 * k + 1];
        ++k;
      }
      if (out > out_row_ptr[u] && out_col[out - 1] == c) continue; /* duplicate pair */
      out_col[out++] = c;
    }
    out_row_ptr[u + 1] = (int32_t)out;
  }
  free(dir);
  return out;
}

/* ---- full solve ----------------------------------------------------------
 * round loop:
 *   GDP phase from the current lambda (F bits) until a fixed point or the cap;
 *   while pricing rounds remain, after the first phase and after any phase
 *     whose preceding scan found at least n/1024 pairs: price with that lambda;
 *     if pairs were found, add them and start the next GDP phase (lambda kept),
 *     except after the first phase's scan when it found fewer than n/1024
 *     pairs: then go on to rule (7) and the finisher, which take the few new
 *     edges from this lambda -- after a scan that found few pairs the next
 *     phase goes straight on, since the scan with the final lambda below finds
 *     what is still missing;
 *   otherwise extract x by rule (7); if a node's row does not sum to 2, run the
 *     exact finisher (lambda then has F+1 bits);
 *   price with the final lambda: no pair -> certified optimal over all pairs;
 *     else add the pairs, continue GDP from lambda (F bits: lambda2 >> 1). */

struct or_result {
  int32_t n;
  int64_t nnz;
  int32_t* row_ptr;
  int32_t* col;
  uint8_t* x2;
  int32_t* lam;
};

static int64_t or_price_all(int32_t n, const int32_t* xy, const int32_t* rp, const int32_t* cl,
                            const int32_t* lam, int32_t fb, int32_t** pairs, int64_t* cap) {
  int64_t cnt = or_pricing(n, xy, rp, cl, lam, fb, *pairs, *cap);
  if (cnt > *cap) {
    free(*pairs);
    *cap = cnt;
    *pairs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * cnt));
    cnt = or_pricing(n, xy, rp, cl, lam, fb, *pairs, *cap);
  }
  return cnt;
}

static void or_add_pairs(or_result* r, const int32_t* xy, int32_t** cost, int64_t npairs,
                         const int32_t* pairs) {
  int32_t* nrp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r->n + 1));
  int32_t* ncl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r->nnz + 2 * npairs));
  int64_t nnz = or_merge(r->n, r->row_ptr, r->col, npairs, pairs, nrp, ncl);
  free(r->row_ptr); free(r->col); free(*cost); free(r->x2);
  r->row_ptr = nrp; r->col = ncl; r->nnz = nnz;
  *cost = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  r->x2 = (uint8_t*)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
  or_cost_table(r->n, xy, r->row_ptr, r->col, *cost);
}

or_result* or_solve(int32_t n, const int32_t* xy, const int32_t* row_ptr,
                    const int32_t* col, const int32_t* b, const int32_t* lam0, const or_params* p,
                    or_info* info, int64_t* trace_bound2, int64_t* trace_changed,
                    int64_t trace_cap) {
  or_result* r = (or_result*)calloc(1, sizeof(or_result));
  r->n = n;
  r->nnz = row_ptr[n];
  r->row_ptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  r->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r->nnz > 0 ? r->nnz : 1));
  memcpy(r->row_ptr, row_ptr, sizeof(int32_t) * (size_t)(n + 1));
  memcpy(r->col, col, sizeof(int32_t) * (size_t)r->nnz);
  r->x2 = (uint8_t*)calloc((size_t)(r->nnz > 0 ? r->nnz : 1), 1);
  r->lam = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int32_t* cost = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r->nnz > 0 ? r->nnz : 1));
  or_cost_table(n, xy, r->row_ptr, r->col, cost);
  int32_t* lam = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int32_t* lam2 = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (lam0) memcpy(lam, lam0, sizeof(int32_t) * (size_t)n);
  int64_t pcap = 1 << 16;
  int32_t* pairs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * pcap));

  const int32_t F = p->frac_bits;
  int64_t last_pairs = 0; /* pairs found by the last scan */
  memset(info, 0, sizeof(*info));
  info->frac_bits = F;
  int status = OR_OK;
  for (;;) {
    int64_t it = 0;
    int64_t off = info->iterations;
    int64_t tcap = trace_cap > off ? trace_cap - off : 0;
    int st;
    if (p->update == OR_UPDATE_CLASSES) {
      /* colour the current graph (pricing may have added edges) */
      int32_t* color = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      int32_t nc = or_color_greedy(n, r->row_ptr, r->col, color);
      st = or_gdp_gs(n, r->row_ptr, r->col, cost, b, color, nc, F, p->damping_shift, p->max_iters,
                     lam, &it, trace_bound2 ? trace_bound2 + off : NULL,
                     trace_changed ? trace_changed + off : NULL, tcap);
      free(color);
    } else {
      st = or_gdp(n, r->row_ptr, r->col, cost, b, F, p->damping_shift, p->max_iters, lam, &it,
                  trace_bound2 ? trace_bound2 + off : NULL,
                  trace_changed ? trace_changed + off : NULL, tcap);
    }
    info->iterations += it;
    info->phases += 1;
    if (st == OR_OVERFLOW || st == OR_INVALID) { status = st; break; }

    int clean = 0; /* the GDP lambda was priced and no pair was found */
    if (p->pricing && info->pricing_rounds < p->max_pricing_rounds &&
        (info->phases == 1 || last_pairs * 1024 >= n)) {
      int64_t cnt = or_price_all(n, xy, r->row_ptr, r->col, lam, F, &pairs, &pcap);
      info->pricing_rounds += 1;
      last_pairs = cnt;
      if (cnt > 0) {
        or_add_pairs(r, xy, &cost, cnt, pairs);
        info->edges_added += cnt;
        /* another GDP phase, unless the first phase's scan found few pairs:
         * the finisher then takes the few new edges from this lambda */
        if (info->phases > 1 || cnt * 1024 >= n) continue;
      } else {
        clean = 1;
      }
    }

    int32_t fb = F;
    int64_t bad = or_extract(n, r->row_ptr, r->col, cost, b, lam, F, r->x2);
    memcpy(r->lam, lam, sizeof(int32_t) * (size_t)n);
    if (bad > 0) {
      if (!p->finisher) { status = OR_NOT_CONVERGED; info->bound2 = or_bound2(n, r->row_ptr, r->col, cost, b, lam, F); break; }
      int64_t aug = 0;
      st = or_finisher(n, r->row_ptr, r->col, cost, b, lam, F, r->x2, lam2, &aug);
      info->finisher_calls += 1;
      info->augmentations += aug;
      if (st != OR_OK) { status = st; break; }
      fb = F + 1;
      memcpy(r->lam, lam2, sizeof(int32_t) * (size_t)n);
    }
    info->frac_bits = fb;
    info->bound2 = or_bound2(n, r->row_ptr, r->col, cost, b, r->lam, fb);
    info->certified = 1;
    if (!p->pricing) break;
    if (fb == F && clean) { info->certified = 2; break; } /* same lambda already priced */
    if (info->pricing_rounds >= p->max_pricing_rounds) { status = OR_NOT_CONVERGED; break; }
    int64_t cnt = or_price_all(n, xy, r->row_ptr, r->col, r->lam, fb, &pairs, &pcap);
    info->pricing_rounds += 1;
    last_pairs = cnt;
    if (cnt == 0) { info->certified = 2; break; }
    or_add_pairs(r, xy, &cost, cnt, pairs);
    info->edges_added += cnt;
    info->certified = 0;
    info->frac_bits = F;
    if (fb == F + 1)
      for (int32_t v = 0; v < n; ++v) lam[v] = r->lam[v] >> 1; /* floor to F bits */
  }
  info->status = status;
  free(cost); free(lam); free(lam2); free(pairs);
  return r;
}

int64_t or_result_nnz(const or_result* r) { return r->nnz; }

void or_result_copy(const or_result* r, int32_t* row_ptr, int32_t* col, uint8_t* x2,
                    int32_t* lam) {
  if (row_ptr) memcpy(row_ptr, r->row_ptr, sizeof(int32_t) * (size_t)(r->n + 1));
  if (col) memcpy(col, r->col, sizeof(int32_t) * (size_t)r->nnz);
  if (x2) memcpy(x2, r->x2, (size_t)r->nnz);
  if (lam) memcpy(lam, r->lam, sizeof(int32_t) * (size_t)r->n);
}

void or_result_free(or_result* r) {
  if (!r) return;
  free(r->row_ptr); free(r->col); free(r->x2); free(r->lam); free(r);
}

/* ---- k nearest neighbours (brute force) ------------------------------------ */

void or_knn(int32_t n, const int32_t* xy, int32_t k, int32_t* nbr, int64_t* d2) {
  for (int32_t i = 0; i < n; ++i) {
    int32_t* bi = nbr + (int64_t)i * k;
    int64_t* bd = d2 + (int64_t)i * k;
    int32_t cnt = 0;
    for (int32_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const int64_t dx = (int64_t)xy[2 * j] - xy[2 * i];
      const int64_t dy = (int64_t)xy[2 * j + 1] - xy[2 * i + 1];
      const int64_t d = dx * dx + dy * dy;
      /* (d, j) belongs in the list if it precedes the current k-th entry */
      if (cnt == k && !(d < bd[k - 1] || (d == bd[k - 1] && j < bi[k - 1]))) continue;
      int32_t p = cnt < k ? cnt++ : k - 1;
      while (p > 0 && (d < bd[p - 1] || (d == bd[p - 1] && j < bi[p - 1]))) {
        bd[p] = bd[p - 1];
        bi[p] = bi[p - 1];
        --p;
      }
      bd[p] = d;
      bi[p] = j;
    }
  }
}
