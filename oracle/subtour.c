/* CPU oracle for GDP with subtour-elimination cuts -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline / reference arm
 * load this code; the CUDA library never does and shares no code with it.
 *
 * The LP (Section 2, LP3 with equalities (1) and inequalities (2); Section 4's
 * F2M plus the subtour elimination constraints that the paper's Discussion
 * names as the next relaxation):
 *   minimise c x  subject to  x(delta(v)) = 2 for every node v,
 *                             x(delta(S)) >= 2 for every cut S of a family,
 *                             0 <= x <= 1.
 * Every constraint has binary coefficients and integral right side 2 (Eq. 8),
 * so Section 3's gradient applies to each: from the 2nd and 3rd smallest
 * modified values over its support.  The inequality duals are kept >= 0
 * (Eq. 5).  The modified objective (Eq. 4) of an edge uv is
 *   z_uv = c_uv 2^F - lambda_u - lambda_v - sum of mu_S over the cuts S with
 *          exactly one of u, v in S.
 *
 * Cut family: L layers; layer l labels every node comp[l n + v] with -1 (in no
 * cut of the layer) or s in [0, ncuts[l]); the nodes labelled s form the cut
 * set S_(l,s).  Cuts of one layer are disjoint sets.  mu holds the cut duals
 * layer after layer (layer l's at mu + sum of ncuts[0..l-1]), units 2^-F.
 *
 * Readings where the paper is silent (each is a stated choice):
 *   - one Jacobi sweep updates every lambda and every mu from the same input
 *     (Section 5.1's parallel update extended to the cut duals):
 *       lambda_v += trunc((z(2) + z(3)) / 2^shift) over delta(v),
 *       mu_S = max(0, mu_S + trunc((z(2) + z(3)) / 2^(shift + 2))) over delta(S);
 *     the cut step is a quarter of the node step, because an edge's z moves
 *     with both end duals and up to two cut duals per layer at once (with the
 *     node-sized step the duals diverged after a few layers on the oracle);
 *   - bound2 = 4 sum lambda + 4 sum mu + sum over directed entries of
 *     min(0, z), twice the Lagrangian bound at the sweep's input;
 *   - a cut needs at least 3 crossing candidate edges (the 3rd value of
 *     Section 3's gradient); separation leaves out components with fewer;
 *   - overflow when some |lambda| or mu reaches 2^29.
 * Separation: the connected components of the support of x (x from rule (7)
 * at the current duals); if there are m >= 3, each is a cut; if m = 2, the one
 * without node 0 (delta(S) = delta(V \ S)); components are numbered by their
 * smallest node.
 */
#include "f2m_oracle.h"

#include <stdlib.h>
#include <string.h>

#define OR_LAM_LIMIT (1LL << 29)

static int cmp_i64s(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* sum over the layers of the cut duals of the cuts that edge (u, v) crosses */
static int64_t or_cut_term(int32_t n, int32_t L, const int32_t* comp, const int32_t* ncuts,
                           const int32_t* mu, int32_t u, int32_t v) {
  int64_t t = 0;
  int64_t off = 0;
  for (int32_t l = 0; l < L; ++l) {
    const int32_t a = comp[(int64_t)l * n + u], b = comp[(int64_t)l * n + v];
    if (a != b) {
      if (a >= 0) t += mu[off + a];
      if (b >= 0) t += mu[off + b];
    }
    off += ncuts[l];
  }
  return t;
}

int64_t or_cut_z(int32_t n, const int32_t* xy, int32_t L, const int32_t* comp, const int32_t* ncuts,
                 const int32_t* lam, const int32_t* mu, int32_t fb, int32_t u, int32_t v) {
  return ((int64_t)or_cost(xy, u, v) << fb) - lam[u] - lam[v] - or_cut_term(n, L, comp, ncuts, mu, u, v);
}

static int64_t or_total_cuts(int32_t L, const int32_t* ncuts) {
  int64_t m = 0;
  for (int32_t l = 0; l < L; ++l) m += ncuts[l];
  return m;
}

int64_t or_cut_bound2(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                      int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam,
                      const int32_t* mu, int32_t fb) {
  int64_t b2 = 0;
  const int64_t M = or_total_cuts(L, ncuts);
  for (int64_t s = 0; s < M; ++s) b2 += 4 * (int64_t)mu[s];
  for (int32_t v = 0; v < n; ++v) {
    b2 += 4 * (int64_t)lam[v];
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int64_t z = ((int64_t)cost[e] << fb) - lam[v] - lam[col[e]] -
                  or_cut_term(n, L, comp, ncuts, mu, v, col[e]);
      if (z < 0) b2 += z;
    }
  }
  return b2;
}

int or_cut_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                 int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam_old,
                 const int32_t* mu_old, int32_t F, int32_t shift, int32_t* lam_new, int32_t* mu_new,
                 int64_t* bound2, int64_t* changed) {
  const int64_t nnz = row_ptr[n];
  const int64_t M = or_total_cuts(L, ncuts);
  int64_t* z = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1)); /* z per entry */
  int64_t b2 = 0, ch = 0;
  int status = OR_OK;
  /* Eq. 4 / Eq. 9 with the cut terms, per directed entry, from the input duals */
  for (int32_t v = 0; v < n; ++v)
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      z[e] = ((int64_t)cost[e] << F) - lam_old[v] - lam_old[col[e]] -
             or_cut_term(n, L, comp, ncuts, mu_old, v, col[e]);
      if (z[e] < 0) b2 += z[e];
    }
  for (int64_t s = 0; s < M; ++s) b2 += 4 * (int64_t)mu_old[s];
  /* node duals: 2nd and 3rd smallest z over delta(v) (Section 3, b = 2) */
  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
  int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxdeg > 0 ? maxdeg : 1));
  for (int32_t v = 0; v < n && status != OR_INVALID; ++v) {
    const int32_t deg = row_ptr[v + 1] - row_ptr[v];
    if (deg < 3) { status = OR_INVALID; break; }
    memcpy(buf, z + row_ptr[v], sizeof(int64_t) * (size_t)deg);
    qsort(buf, (size_t)deg, sizeof(int64_t), cmp_i64s);
    const int64_t d = (buf[1] + buf[2]) / ((int64_t)1 << shift); /* toward zero */
    const int64_t nl = (int64_t)lam_old[v] + d;
    if (nl >= OR_LAM_LIMIT || nl <= -OR_LAM_LIMIT) status = OR_OVERFLOW;
    lam_new[v] = (int32_t)nl;
    b2 += 4 * (int64_t)lam_old[v];
    if (d != 0) ++ch;
  }
  free(buf);
  /* cut duals: 2nd and 3rd smallest z over delta(S); each crossing edge once,
   * from the entry whose row lies in S; projected onto mu >= 0 (Eq. 5) */
  int64_t off = 0;
  for (int32_t l = 0; l < L && status != OR_INVALID; ++l) {
    const int32_t* cl = comp + (int64_t)l * n;
    int64_t* cnt = (int64_t*)calloc((size_t)ncuts[l] + 1, sizeof(int64_t));
    for (int32_t u = 0; u < n; ++u) {
      if (cl[u] < 0) continue;
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
        if (cl[col[e]] != cl[u]) ++cnt[cl[u] + 1];
    }
    for (int32_t s = 0; s < ncuts[l]; ++s) cnt[s + 1] += cnt[s];
    int64_t* vals = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cnt[ncuts[l]] > 0 ? cnt[ncuts[l]] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncuts[l] > 0 ? ncuts[l] : 1));
    for (int32_t s = 0; s < ncuts[l]; ++s) fill[s] = cnt[s];
    for (int32_t u = 0; u < n; ++u) {
      if (cl[u] < 0) continue;
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
        if (cl[col[e]] != cl[u]) vals[fill[cl[u]]++] = z[e];
    }
    for (int32_t s = 0; s < ncuts[l]; ++s) {
      const int64_t k = cnt[s + 1] - cnt[s];
      if (k < 3) { status = OR_INVALID; break; }
      qsort(vals + cnt[s], (size_t)k, sizeof(int64_t), cmp_i64s);
      const int64_t d = (vals[cnt[s] + 1] + vals[cnt[s] + 2]) / ((int64_t)1 << (shift + 2));
      int64_t nm = (int64_t)mu_old[off + s] + d;
      if (nm < 0) nm = 0;
      if (nm >= OR_LAM_LIMIT) status = OR_OVERFLOW;
      mu_new[off + s] = (int32_t)nm;
      if (nm != mu_old[off + s]) ++ch;
    }
    free(cnt); free(vals); free(fill);
    off += ncuts[l];
  }
  free(z);
  *bound2 = b2;
  *changed = ch;
  return status;
}

int or_cut_gdp(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost, int32_t L,
               const int32_t* comp, const int32_t* ncuts, int32_t F, int32_t shift, int64_t max_iters,
               int32_t* lam, int32_t* mu, int64_t* iters, int64_t* trace_bound2, int64_t* trace_changed,
               int64_t trace_cap) {
  const int64_t M = or_total_cuts(L, ncuts);
  int32_t* nl = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* nm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  int status = OR_NOT_CONVERGED;
  int64_t it = 0;
  while (it < max_iters) {
    int64_t b2, ch;
    int st = or_cut_sweep(n, row_ptr, col, cost, L, comp, ncuts, lam, mu, F, shift, nl, nm, &b2, &ch);
    if (it < trace_cap) {
      if (trace_bound2) trace_bound2[it] = b2;
      if (trace_changed) trace_changed[it] = ch;
    }
    ++it;
    if (st != OR_OK) { status = st; break; }
    memcpy(lam, nl, sizeof(int32_t) * (size_t)n);
    if (M > 0) memcpy(mu, nm, sizeof(int32_t) * (size_t)M);
    if (ch == 0) { status = OR_OK; break; }
  }
  free(nl); free(nm);
  *iters = it;
  return status;
}

int64_t or_cut_extract(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* cost,
                       int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam,
                       const int32_t* mu, int32_t fb, uint8_t* x2) {
  int64_t bad = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t s = 0;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int64_t z = ((int64_t)cost[e] << fb) - lam[v] - lam[col[e]] -
                  or_cut_term(n, L, comp, ncuts, mu, v, col[e]);
      x2[e] = (uint8_t)(z < 0 ? 2 : (z == 0 ? 1 : 0));
      s += x2[e];
    }
    if (s != 4) ++bad;
  }
  return bad;
}

int32_t or_separate(int32_t n, const int32_t* row_ptr, const int32_t* col, const uint8_t* x2,
                    int32_t* comp) {
  /* components of the support {e : x2_e > 0}, by depth-first search from the
   * nodes in ascending order: component k is the one whose smallest node is
   * the k-th smallest of the components' smallest nodes */
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* id = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t v = 0; v < n; ++v) id[v] = -1;
  int32_t m = 0;
  for (int32_t r = 0; r < n; ++r) {
    if (id[r] >= 0) continue;
    int32_t sp = 0;
    stack[sp++] = r;
    id[r] = m;
    while (sp > 0) {
      int32_t u = stack[--sp];
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
        if (x2[e] > 0 && id[col[e]] < 0) { id[col[e]] = m; stack[sp++] = col[e]; }
    }
    ++m;
  }
  /* crossing candidate edges per component (each edge counted from both sides) */
  int64_t* cross = (int64_t*)calloc((size_t)m, sizeof(int64_t));
  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (id[col[e]] != id[u]) ++cross[id[u]];
  /* the cuts: every component if m >= 3, the one without node 0 if m = 2;
   * left out if fewer than 3 candidate edges cross it */
  int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t ncut = 0;
  for (int32_t k = 0; k < m; ++k) {
    int take = m >= 3 || (m == 2 && k != id[0]);
    lab[k] = (take && cross[k] >= 3) ? ncut++ : -1;
  }
  for (int32_t v = 0; v < n; ++v) comp[v] = m >= 2 ? lab[id[v]] : -1;
  free(stack); free(id); free(cross); free(lab);
  return ncut;
}

int64_t or_cut_pricing(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
                       int32_t L, const int32_t* comp, const int32_t* ncuts, const int32_t* lam,
                       const int32_t* mu, int32_t fb, int32_t* pairs, int64_t cap) {
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) mark[v] = -1;
  int64_t count = 0;
  for (int32_t u = 0; u < n; ++u) {
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) mark[col[e]] = u;
    for (int32_t v = u + 1; v < n; ++v) {
      if (mark[v] == u) continue;
      if (or_cut_z(n, xy, L, comp, ncuts, lam, mu, fb, u, v) < 0) {
        if (count < cap) { pairs[2 * count] = u; pairs[2 * count + 1] = v; }
        ++count;
      }
    }
  }
  free(mark);
  return count;
}

/* ---- the driver: stages of GDP with pricing, cut layers between them -------
 * A stage: a GDP phase (or_cut_gdp, at most max_iters sweeps); then a pricing
 * scan with the cut terms; while it finds pairs they are merged (costs
 * recomputed) and another phase runs; the stage ends with rule (7) x and the
 * bound at the duals reached.  Stage 0 runs without cuts (the F2M GDP); each
 * of the next `rounds` stages first adds the layer or_separate makes from the
 * previous stage's x, and the rounds stop early when it makes no cut. */

struct or_subtour {
  int32_t n;
  int64_t nnz;
  int32_t* row_ptr;
  int32_t* col;
  uint8_t* x2;
  int32_t* lam;
  int32_t L;
  int32_t ncuts[8];
  int32_t* comp;  /* [8][n] */
  int32_t* mu;
  int64_t M;
};

int64_t or_subtour_nnz(const or_subtour* r) { return r->nnz; }
int64_t or_subtour_cuts(const or_subtour* r) { return r->M; }
int32_t or_subtour_layers(const or_subtour* r) { return r->L; }

void or_subtour_copy(const or_subtour* r, int32_t* row_ptr, int32_t* col, uint8_t* x2, int32_t* lam,
                     int32_t* mu, int32_t* comp, int32_t* ncuts) {
  if (row_ptr) memcpy(row_ptr, r->row_ptr, sizeof(int32_t) * (size_t)(r->n + 1));
  if (col) memcpy(col, r->col, sizeof(int32_t) * (size_t)r->nnz);
  if (x2) memcpy(x2, r->x2, (size_t)r->nnz);
  if (lam) memcpy(lam, r->lam, sizeof(int32_t) * (size_t)r->n);
  if (mu && r->M) memcpy(mu, r->mu, sizeof(int32_t) * (size_t)r->M);
  if (comp && r->L) memcpy(comp, r->comp, sizeof(int32_t) * (size_t)r->L * r->n);
  if (ncuts && r->L) memcpy(ncuts, r->ncuts, sizeof(int32_t) * (size_t)r->L);
}

void or_subtour_free(or_subtour* r) {
  if (!r) return;
  free(r->row_ptr); free(r->col); free(r->x2); free(r->lam); free(r->comp); free(r->mu); free(r);
}

/* one stage; returns an OR_ status */
static int or_stage(or_subtour* r, const int32_t* xy, int32_t** cost, int32_t F, int32_t shift,
                    int64_t max_iters, int32_t pricing, int32_t max_pricing_rounds, or_subtour_info* info,
                    int64_t* bound2) {
  const int32_t n = r->n;
  for (;;) {
    int64_t it = 0;
    int st = or_cut_gdp(n, r->row_ptr, r->col, *cost, r->L, r->comp, r->ncuts, F, shift, max_iters, r->lam,
                        r->mu, &it, NULL, NULL, 0);
    info->iterations += it;
    info->phases += 1;
    if (st != OR_OK && st != OR_NOT_CONVERGED) return st;
    if (!pricing) break;
    if (info->pricing_rounds >= max_pricing_rounds) return OR_NOT_CONVERGED;
    int64_t cnt = or_cut_pricing(n, xy, r->row_ptr, r->col, r->L, r->comp, r->ncuts, r->lam, r->mu, F, NULL, 0);
    int32_t* pairs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * cnt + 2));
    or_cut_pricing(n, xy, r->row_ptr, r->col, r->L, r->comp, r->ncuts, r->lam, r->mu, F, pairs, cnt);
    info->pricing_rounds += 1;
    if (cnt == 0) { free(pairs); break; }
    int32_t* nrp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t* ncl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r->nnz + 2 * cnt));
    int64_t nnz = or_merge(n, r->row_ptr, r->col, cnt, pairs, nrp, ncl);
    free(pairs);
    free(r->row_ptr); free(r->col); free(*cost); free(r->x2);
    r->row_ptr = nrp; r->col = ncl; r->nnz = nnz;
    *cost = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    r->x2 = (uint8_t*)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
    or_cost_table(n, xy, r->row_ptr, r->col, *cost);
    info->edges_added += cnt;
  }
  or_cut_extract(n, r->row_ptr, r->col, *cost, r->L, r->comp, r->ncuts, r->lam, r->mu, F, r->x2);
  *bound2 = or_cut_bound2(n, r->row_ptr, r->col, *cost, r->L, r->comp, r->ncuts, r->lam, r->mu, F);
  return OR_OK;
}

or_subtour* or_solve_subtour(int32_t n, const int32_t* xy, const int32_t* row_ptr, const int32_t* col,
                             const int32_t* lam0, int32_t F, int32_t shift, int64_t max_iters,
                             int32_t pricing, int32_t max_pricing_rounds, int32_t rounds,
                             or_subtour_info* info) {
  or_subtour* r = (or_subtour*)calloc(1, sizeof(or_subtour));
  r->n = n;
  r->nnz = row_ptr[n];
  r->row_ptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  r->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r->nnz > 0 ? r->nnz : 1));
  memcpy(r->row_ptr, row_ptr, sizeof(int32_t) * (size_t)(n + 1));
  memcpy(r->col, col, sizeof(int32_t) * (size_t)r->nnz);
  r->x2 = (uint8_t*)calloc((size_t)(r->nnz > 0 ? r->nnz : 1), 1);
  r->lam = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (lam0) memcpy(r->lam, lam0, sizeof(int32_t) * (size_t)n);
  r->comp = (int32_t*)malloc(sizeof(int32_t) * (size_t)8 * n);
  r->mu = NULL;
  int32_t* cost = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r->nnz > 0 ? r->nnz : 1));
  or_cost_table(n, xy, r->row_ptr, r->col, cost);
  memset(info, 0, sizeof(*info));
  info->frac_bits = F;
  int64_t b2 = 0;
  int st = or_stage(r, xy, &cost, F, shift, max_iters, pricing, max_pricing_rounds, info, &b2);
  info->bound2_f2m = b2;
  info->bound2 = b2;
  int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t k = 0; k < rounds && st == OR_OK && r->L < 8; ++k) {
    int32_t m = or_separate(n, r->row_ptr, r->col, r->x2, lab);
    if (m == 0) break;
    memcpy(r->comp + (int64_t)r->L * n, lab, sizeof(int32_t) * (size_t)n);
    r->ncuts[r->L] = m;
    r->L += 1;
    r->mu = (int32_t*)realloc(r->mu, sizeof(int32_t) * (size_t)(r->M + m));
    memset(r->mu + r->M, 0, sizeof(int32_t) * (size_t)m);
    r->M += m;
    info->rounds += 1;
    info->cuts += m;
    st = or_stage(r, xy, &cost, F, shift, max_iters, pricing, max_pricing_rounds, info, &b2);
    info->bound2 = b2;
  }
  free(lab);
  free(cost);
  info->layers = r->L;
  info->certified = (st == OR_OK && pricing) ? 1 : 0;
  info->status = st;
  return r;
}
