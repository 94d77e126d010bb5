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
// lowest-numbered node with surplus to the nearest node with deficit (Dijkstra
// on reduced costs, heap order (distance, node)), and raise pi by
// d(t) - d(i) on the nodes settled before t.  The rules are fixed, so the
// result is deterministic.
#include <cstdint>
#include <queue>
#include <utility>
#include <vector>

#include "f2m_internal.h"

namespace f2m {

namespace {

struct Network {
  int32_t n = 0;
  int64_t m = 0;
  std::vector<int32_t> head_of;   // per arc: v of L_u -> R_v
  std::vector<int32_t> tail_of;   // per arc: u
  std::vector<int64_t> cost;      // per arc: c * 2^F
  std::vector<int32_t> twin;      // per arc: the arc of the opposite direction (v -> u)
  std::vector<uint8_t> flow;      // per arc: 0 or 1
  std::vector<int32_t> off;       // CSR offsets shared by L_u (out arcs) and R_u (in arcs)
};

}  // namespace

int host_finisher(int32_t n, const int32_t* rp, const int2* ec, const int32_t* lam, int32_t F,
                  uint8_t* x2, int32_t* lam2, int64_t* augmentations) {
  Network g;
  g.n = n;
  g.m = rp[n];
  g.off.assign(rp, rp + n + 1);
  g.head_of.resize(g.m);
  g.tail_of.resize(g.m);
  g.cost.resize(g.m);
  g.twin.resize(g.m);
  g.flow.assign(g.m, 0);
  for (int32_t u = 0; u < n; ++u) {
    for (int32_t a = rp[u]; a < rp[u + 1]; ++a) {
      g.head_of[a] = ec[a].x;
      g.tail_of[a] = u;
      g.cost[a] = (int64_t)ec[a].y << F;
    }
  }
  // twin arcs: rows are sorted, so walk row v for each u in increasing order
  {
    std::vector<int32_t> pos(g.off.begin(), g.off.end() - 1);
    for (int32_t u = 0; u < n; ++u) {
      for (int32_t a = rp[u]; a < rp[u + 1]; ++a) {
        const int32_t v = g.head_of[a];
        // entries of row v are visited in increasing u, which is their column order
        int32_t b = pos[v];
        while (b < rp[v + 1] && g.head_of[b] < u) ++b;
        if (b >= rp[v + 1] || g.head_of[b] != u) return 1;  // not symmetric
        g.twin[a] = b;
        pos[v] = b + 1;
      }
    }
  }
  const int32_t N = 2 * n;  // node ids: L_v = v, R_v = n + v
  std::vector<int64_t> pi(N), excess(N);
  for (int32_t v = 0; v < n; ++v) {
    pi[v] = lam[v];
    pi[n + v] = -(int64_t)lam[v];
  }
  std::vector<int32_t> outflow(n, 0), inflow(n, 0);
  for (int64_t a = 0; a < g.m; ++a) {
    const int64_t z = g.cost[a] - lam[g.tail_of[a]] - lam[g.head_of[a]];
    if (z < 0) {
      g.flow[a] = 1;
      ++outflow[g.tail_of[a]];
      ++inflow[g.head_of[a]];
    }
  }
  for (int32_t v = 0; v < n; ++v) {
    excess[v] = 2 - outflow[v];
    excess[n + v] = inflow[v] - 2;
  }

  std::vector<int64_t> dist(N);
  std::vector<int32_t> via(N);            // arc used to reach the node
  std::vector<uint32_t> reached(N, 0), closed(N, 0);
  std::vector<int32_t> order;
  order.reserve(1024);
  typedef std::pair<int64_t, int32_t> Item;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
  uint32_t round = 0;
  int64_t pushes = 0;
  int32_t next_src = 0;
  int status = 0;

  for (;;) {
    while (next_src < N && excess[next_src] <= 0) ++next_src;
    if (next_src >= N) break;
    const int32_t s = next_src;
    ++round;
    order.clear();
    while (!pq.empty()) pq.pop();
    dist[s] = 0;
    reached[s] = round;
    via[s] = -1;
    pq.push(Item(0, s));
    int32_t t = -1;
    while (!pq.empty()) {
      const Item top = pq.top();
      pq.pop();
      const int32_t i = top.second;
      if (closed[i] == round || top.first != dist[i]) continue;
      closed[i] = round;
      if (excess[i] < 0) { t = i; break; }
      order.push_back(i);
      if (i < n) {
        // out arcs of L_i with no flow: L_i -> R_head
        for (int32_t a = g.off[i]; a < g.off[i + 1]; ++a) {
          if (g.flow[a]) continue;
          const int32_t j = n + g.head_of[a];
          const int64_t d = dist[i] + g.cost[a] - pi[i] + pi[j];
          if (closed[j] != round && (reached[j] != round || d < dist[j])) {
            reached[j] = round; dist[j] = d; via[j] = a;
            pq.push(Item(d, j));
          }
        }
      } else {
        // R_v: reverse arcs of saturated arcs u -> v, i.e. the twins of row v
        const int32_t v = i - n;
        for (int32_t b = g.off[v]; b < g.off[v + 1]; ++b) {
          const int32_t a = g.twin[b];  // arc (head_of[b] -> v)
          if (!g.flow[a]) continue;
          const int32_t j = g.tail_of[a];
          const int64_t d = dist[i] - g.cost[a] - pi[i] + pi[j];
          if (closed[j] != round && (reached[j] != round || d < dist[j])) {
            reached[j] = round; dist[j] = d; via[j] = a;
            pq.push(Item(d, j));
          }
        }
      }
    }
    if (t < 0) { status = 7; break; }
    for (int32_t j = t; j != s;) {
      const int32_t a = via[j];
      if (j >= n) { g.flow[a] = 1; j = g.tail_of[a]; }
      else { g.flow[a] = 0; j = n + g.head_of[a]; }
    }
    excess[s] -= 1;
    excess[t] += 1;
    ++pushes;
    const int64_t dt = dist[t];
    for (int32_t i : order) pi[i] += dt - dist[i];
  }
  *augmentations = pushes;
  if (status != 0) return status;
  for (int64_t a = 0; a < g.m; ++a) x2[a] = (uint8_t)(g.flow[a] + g.flow[g.twin[a]]);
  for (int32_t v = 0; v < n; ++v) {
    const int64_t l2 = pi[v] - pi[n + v];
    if (l2 >= 2 * kLamLimit || l2 <= -2 * kLamLimit) status = 5;
    lam2[v] = (int32_t)l2;
  }
  return status;
}

}  // namespace f2m
