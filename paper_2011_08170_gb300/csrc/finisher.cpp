// Exact finisher (host): min-cost flow on the bipartite double cover.
//
// Section 3 (last paragraph) notes that the gradient procedure does not control
// the constraint values and can stop where the sign rule (7) gives a point that
// violates some constraints by +-1, 2, ..., leaving the repair to problem-
// specific means.  For F2M the repair is exact: the fractional 2-matching LP on
// a graph equals half of the bipartite 2-matching (transportation) problem on
// its double cover, with a left copy L_v (supply 2) and a right copy R_v
// (demand 2) of every node and, for every directed CSR entry u -> v, an arc
// L_u -> R_v of capacity 1 and cost C = c_uv * 2^F.  From an optimal flow y and
// optimal potentials pi:  x_uv = (y(L_u R_v) + y(L_v R_u)) / 2  and
// lambda_v = (pi(L_v) - pi(R_v)) / 2 are optimal for F2M (the latter is
// returned in units 2^-(F+1) as pi(L_v) - pi(R_v)).
//
// Warm start from the GDP duals: pi(L_v) = lambda_v, pi(R_v) = -lambda_v, so an
// arc's reduced cost C - pi(tail) + pi(head) is the adjusted length z_e (Eq. 9);
// arcs with z_e < 0 start saturated, so no residual arc has negative reduced
// cost.  Successive shortest paths then move one unit per step from the
// surplus node with the smallest key to the nearest node with deficit
// (Dijkstra on reduced costs, heap order (distance, key)), and raise pi by
// d(t) - d(i) on the nodes settled before t.  The key orders nodes along a
// Morton curve of their points (ties by caller id), left copy before right
// copy, so successive searches stay in nearby memory.  The rules are fixed,
// so the result is deterministic.
//
// Layout: the graph arrives in the renumbered node order prepared on the
// device (finisher_prep.cu): internal node i is the i-th point in (Morton
// code, caller id) order, every row keeps the caller's column order.  Node
// ids here: L_i = i, R_i = n + i; key(L_i) = 2i, key(R_i) = 2i + 1.
#include <cstdint>
#include <vector>

#include "f2m_internal.h"

namespace f2m {

struct FinisherWork {
  std::vector<int64_t> pi, dist;
  std::vector<int32_t> excess, via, pred, order;
  std::vector<int32_t> sources;  // surplus nodes in key order
  std::vector<uint32_t> reached, closed;
  uint32_t round = 0;
  struct Item {
    int64_t d;
    int32_t key;   // the tie-break
    int32_t node;  // internal id
  };
  std::vector<Item> heap;

  static bool less(const Item& a, const Item& b) { return a.d < b.d || (a.d == b.d && a.key < b.key); }
  void push(const Item& it) {
    heap.push_back(it);
    size_t i = heap.size() - 1;
    while (i > 0) {
      const size_t p = (i - 1) / 2;
      if (!less(heap[i], heap[p])) break;
      const Item t = heap[i]; heap[i] = heap[p]; heap[p] = t;
      i = p;
    }
  }
  Item pop() {
    const Item top = heap[0];
    heap[0] = heap.back();
    heap.pop_back();
    size_t i = 0;
    const size_t m = heap.size();
    for (;;) {
      const size_t l = 2 * i + 1, r = l + 1;
      size_t s = i;
      if (l < m && less(heap[l], heap[s])) s = l;
      if (r < m && less(heap[r], heap[s])) s = r;
      if (s == i) break;
      const Item t = heap[i]; heap[i] = heap[s]; heap[s] = t;
      i = s;
    }
    return top;
  }
};

FinisherWork* finisher_work_new() { return new FinisherWork(); }

void finisher_work_reserve(FinisherWork* w, int32_t n) {
  const size_t N = 2 * (size_t)n;
  if (w->pi.size() >= N) return;
  w->pi.assign(N, 0);
  w->dist.assign(N, 0);
  w->excess.assign(N, 0);
  w->via.assign(N, 0);
  w->pred.assign(N, 0);
  w->reached.assign(N, 0);
  w->closed.assign(N, 0);
  w->round = 0;
  w->order.reserve(1024);
  w->heap.reserve(4096);
  w->sources.reserve(N / 16 + 64);
}
void finisher_work_free(FinisherWork* w) { delete w; }

int host_finisher(int32_t n, const int32_t* irp, const int2* iec, const int32_t* twin, uint8_t* y,
                  const int32_t* exl, const int32_t* lam, int32_t F, uint8_t* x2, int32_t* lam2,
                  int64_t* augmentations, FinisherWork* w) {
  const int32_t N = 2 * n;
  finisher_work_reserve(w, n);
  int64_t* pi = w->pi.data();
  int64_t* dist = w->dist.data();
  int32_t* excess = w->excess.data();
  int32_t* via = w->via.data();
  int32_t* pred = w->pred.data();
  uint32_t* reached = w->reached.data();
  uint32_t* closed = w->closed.data();
  for (int32_t i = 0; i < n; ++i) {
    pi[i] = lam[i];
    pi[n + i] = -(int64_t)lam[i];
    excess[i] = exl[i];       // L_i: supply 2 minus outflow
    excess[n + i] = -exl[i];  // R_i: inflow minus demand 2 (z is symmetric)
  }
  auto key_of = [&](int32_t node) { return node < n ? 2 * node : 2 * (node - n) + 1; };

  // Surplus only shrinks (a path ends at a deficit node), so the nodes that
  // will ever be sources are those with surplus now, taken in key order, each
  // until its surplus is used up.
  std::vector<int32_t>& src = w->sources;
  src.clear();
  for (int32_t i = 0; i < n; ++i) {
    if (excess[i] > 0) src.push_back(i);
    if (excess[n + i] > 0) src.push_back(n + i);
  }

  int64_t pushes = 0;
  int status = 0;
  size_t next_src = 0;
  for (;;) {
    int32_t s = -1;
    while (next_src < src.size()) {
      const int32_t node = src[next_src];
      if (excess[node] > 0) { s = node; break; }
      ++next_src;
    }
    if (s < 0) break;
    if (++w->round == 0) {  // stamp wrap: clear and restart
      w->reached.assign(N, 0);
      w->closed.assign(N, 0);
      w->round = 1;
    }
    const uint32_t round = w->round;
    w->order.clear();
    w->heap.clear();
    dist[s] = 0;
    reached[s] = round;
    pred[s] = -1;
    w->push({0, key_of(s), s});
    int32_t t = -1;
    while (!w->heap.empty()) {
      const FinisherWork::Item top = w->pop();
      const int32_t i = top.node;
      if (closed[i] == round || top.d != dist[i]) continue;
      closed[i] = round;
      if (excess[i] < 0) { t = i; break; }
      w->order.push_back(i);
      if (i < n) {
        // out arcs of L_i without flow: L_i -> R_j
        for (int32_t e = irp[i]; e < irp[i + 1]; ++e) {
          if (y[e]) continue;
          const int32_t j = n + iec[e].x;
          const int64_t d = dist[i] + ((int64_t)iec[e].y << F) - pi[i] + pi[j];
          if (closed[j] != round && (reached[j] != round || d < dist[j])) {
            reached[j] = round; dist[j] = d; via[j] = e; pred[j] = i;
            w->push({d, key_of(j), j});
          }
        }
      } else {
        // R_v: reverse arcs of saturated arcs u -> v (the twins of row v)
        const int32_t v = i - n;
        for (int32_t f = irp[v]; f < irp[v + 1]; ++f) {
          const int32_t a = twin[f];
          if (!y[a]) continue;
          const int32_t j = iec[f].x;  // L_u, the tail of arc a
          const int64_t d = dist[i] - ((int64_t)iec[f].y << F) - pi[i] + pi[j];
          if (closed[j] != round && (reached[j] != round || d < dist[j])) {
            reached[j] = round; dist[j] = d; via[j] = a; pred[j] = i;
            w->push({d, key_of(j), j});
          }
        }
      }
    }
    if (t < 0) { status = 7; break; }
    for (int32_t j = t; j != s; j = pred[j]) y[via[j]] = (uint8_t)(j >= n);  // push one unit
    excess[s] -= 1;
    excess[t] += 1;
    ++pushes;
    const int64_t dt = dist[t];
    for (int32_t i : w->order) pi[i] += dt - dist[i];
  }
  *augmentations = pushes;
  if (status != 0) return status;
  const int64_t nnz = irp[n];
  for (int64_t e = 0; e < nnz; ++e) x2[e] = (uint8_t)(y[e] + y[twin[e]]);
  for (int32_t i = 0; i < n; ++i) {
    const int64_t l2 = pi[i] - pi[n + i];
    if (l2 >= 2 * kLamLimit || l2 <= -2 * kLamLimit) status = 5;
    lam2[i] = (int32_t)l2;
  }
  return status;
}

}  // namespace f2m
