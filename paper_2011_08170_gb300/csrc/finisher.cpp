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
// returned in units 2^-(F+1) as pi(L_v) - pi(R_v)).  With degree requirements
// b_v (fractional b-matching) the supplies and demands are b_v; the caller's
// surpluses exl carry them, so nothing here depends on the value 2.
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
// Three phases.  A blocked phase splits every segment into blocks of B nodes
// (consecutive internal ids, both copies) and runs the blocks on worker
// threads: a block's sources in key order, each search restricted to the
// block -- when a heap item of an outside node comes to the top, or the heap
// runs dry, the search is dropped with nothing changed and the block moves to
// its next source -- with arcs into outside nodes priced at the potentials of
// the phase's start.  Potentials only grow, so every residual reduced cost
// stays non-negative; the arcs and potentials a block reads are written by
// that block alone, so the result does not depend on the schedule.  Phase 1 is
// blocked with B = kFinBlock, phase 2 with B = kFinBlock2 for the searches
// phase 1 dropped (they cross a small block's edge), and phase 3 runs the
// plain search per segment for what is left.
//
// Layout: the graph arrives in the renumbered node order prepared on the
// device (finisher_prep.cu): internal node i is the i-th point in (Morton
// code, caller id) order, every row keeps the caller's column order.  Node
// ids here: L_i = i, R_i = n + i; key(L_i) = 2i, key(R_i) = 2i + 1.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <climits>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "f2m_internal.h"

namespace f2m {

// Search state of one worker: heap, settled list and visit stamps.
struct Searcher {
  struct Item {
    int64_t d;
    int32_t key;   // the tie-break
    int32_t node;  // internal id
  };
  std::vector<Item> heap;
  std::vector<int32_t> order;
  uint32_t stamp_next = 0, stamp_end = 0;  // this worker's unused visit stamps [next, end)

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

constexpr int32_t kFinBlock = kFinBlockNodes;  // nodes per phase-1 block
constexpr int32_t kFinBlock2 = 16384;  // nodes per phase-2 block
constexpr uint32_t kStampChunk = 1024;  // visit stamps a worker takes at a time

// Worker threads kept for the life of the process (one pool, shared by every
// context; jobs from different host threads take turns): a job is a count of
// items handed out by an atomic counter to the calling thread and the workers.
struct WorkerPool {
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_job, cv_done;
  uint64_t generation = 0;  // bumped for every job
  int32_t busy = 0;         // workers still on the current job
  bool quit = false;
  std::function<void(int32_t)> job;  // runs as worker k (k >= 1)
  int32_t job_workers = 0;           // workers 1 .. job_workers - 1 take part

  void start(int32_t nw) {  // nw - 1 threads (the caller is worker 0)
    for (int32_t k = (int32_t)threads.size() + 1; k < nw; ++k)
      threads.emplace_back([this, k] {
        uint64_t seen = 0;
        for (;;) {
          std::function<void(int32_t)> fn;
          {
            std::unique_lock<std::mutex> lk(mu);
            cv_job.wait(lk, [&] { return quit || generation != seen; });
            if (quit) return;
            seen = generation;
            if (k >= job_workers) continue;
            fn = job;
          }
          fn(k);
          std::lock_guard<std::mutex> lk(mu);
          if (--busy == 0) cv_done.notify_all();
        }
      });
  }
  void run(int32_t nw, const std::function<void(int32_t)>& fn) {
    start(nw);
    {
      std::lock_guard<std::mutex> lk(mu);
      job = fn;
      job_workers = nw;
      busy = nw - 1;
      ++generation;
    }
    cv_job.notify_all();
    fn(0);
    std::unique_lock<std::mutex> lk(mu);
    cv_done.wait(lk, [&] { return busy == 0; });
    job = nullptr;
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(mu);
      quit = true;
    }
    cv_job.notify_all();
    for (std::thread& t : threads) t.join();
  }
};

struct FinisherWork {
  int64_t* pi_p = nullptr;    // the potentials in use: pi.data(), or the caller's
  int32_t* ex_p = nullptr;    // the surpluses in use: excess.data(), or the caller's
  std::vector<int64_t> pi, dist;
  std::vector<int64_t> pi_start;  // potentials at phase 2's start (outside nodes are priced with them)
  std::vector<int32_t> excess, via, pred;
  std::vector<uint32_t> reached, closed;  // search stamps; every search takes a fresh one
  std::atomic<uint32_t> stamp{0};
  std::vector<Searcher> workers;
};

WorkerPool& worker_pool() {
  static WorkerPool pool;
  return pool;
}
std::mutex g_pool_turn;  // one job at a time

FinisherWork* finisher_work_new() { return new FinisherWork(); }
void finisher_work_free(FinisherWork* w) { delete w; }

void finisher_work_reserve(FinisherWork* w, int32_t n) {
  const size_t N = 2 * (size_t)n;
  if (w->pi.size() >= N) return;
  w->pi.assign(N, 0);
  w->pi_start.assign(N, 0);
  w->dist.assign(N, 0);
  w->excess.assign(N, 0);
  w->via.assign(N, 0);
  w->pred.assign(N, 0);
  w->reached.assign(N, 0);
  w->closed.assign(N, 0);
  w->stamp.store(0);
}

namespace {

// Successive shortest paths for the sources of nodes [lo, hi) (internal ids),
// in key order.  lam0 == nullptr and pi0 == nullptr: [lo, hi) is a whole
// segment, which no arc leaves (phase 3).  Otherwise [lo, hi) is a block of a
// blocked phase: outside nodes are priced with their potentials at the
// phase's start -- lam0 for a left copy and -lam0 for a right one in phase 1,
// pi0 in phase 2 -- and never settled, and a search that would settle one (or
// finds nothing) is dropped.
// srcs (NULL: every node of [lo, hi)): the nodes that may hold a surplus, in
// key order -- the others are skipped without a look.
int solve_range(int32_t n, int32_t lo, int32_t hi, const int32_t* lam0, const int64_t* pi0v,
                const int32_t* irp, const int2* iec, const int32_t* twin, uint8_t* y, int32_t F,
                FinisherWork* w, Searcher& sr, int64_t* pushes_out, const int32_t* srcs = nullptr,
                int64_t nsrc = 0) {
  int64_t* pi = w->pi_p;
  int64_t* dist = w->dist.data();
  int32_t* excess = w->ex_p;
  int32_t* via = w->via.data();
  int32_t* pred = w->pred.data();
  uint32_t* reached = w->reached.data();
  uint32_t* closed = w->closed.data();
  auto key_of = [&](int32_t node) { return node < n ? 2 * node : 2 * (node - n) + 1; };
  auto outside = [&](int32_t node) {
    const int32_t i = node < n ? node : node - n;
    return i < lo || i >= hi;
  };
  const bool blocked = lam0 || pi0v;
  auto pi0 = [&](int32_t node) {
    if (pi0v) return pi0v[node];
    return node < n ? (int64_t)lam0[node] : -(int64_t)lam0[node - n];
  };
  int64_t pushes = 0;
  const int64_t nitems = srcs ? nsrc : 2LL * (hi - lo);
  for (int64_t item = 0; item < nitems; ++item) {
    {
      // key order: L_i (2i) before R_i (2i+1)
      const int32_t s = srcs ? srcs[item] : ((item & 1) ? n + lo + (int32_t)(item >> 1) : lo + (int32_t)(item >> 1));
      while (excess[s] > 0) {
        if (sr.stamp_next == sr.stamp_end) {  // a fresh chunk of stamps, unique across workers
          sr.stamp_next = w->stamp.fetch_add(kStampChunk) + 1;
          sr.stamp_end = sr.stamp_next + kStampChunk;
        }
        const uint32_t round = sr.stamp_next++;
        sr.order.clear();
        sr.heap.clear();
        dist[s] = 0;
        reached[s] = round;
        pred[s] = -1;
        sr.push({0, key_of(s), s});
        int32_t t = -1;
        // the smallest distance at which a node with deficit has been reached:
        // an item farther than that can never come to the top before the
        // search ends, so it is not pushed (the search is unchanged)
        int64_t bound = INT64_MAX;
        auto note = [&](int32_t j, int64_t d) {
          if (excess[j] < 0 && d < bound) bound = d;
        };
        while (!sr.heap.empty()) {
          const Searcher::Item top = sr.pop();
          const int32_t v = top.node;
          if (blocked && outside(v)) break;  // dropped
          if (closed[v] == round || top.d != dist[v]) continue;
          closed[v] = round;
          if (excess[v] < 0) { t = v; break; }
          sr.order.push_back(v);
          if (v < n) {
            // out arcs of L_v without flow: L_v -> R_j
            for (int32_t e = irp[v]; e < irp[v + 1]; ++e) {
              if (y[e]) continue;
              const int32_t j = n + iec[e].x;
              if (blocked && outside(j)) {
                const int64_t d = dist[v] + ((int64_t)iec[e].y << F) - pi[v] + pi0(j);
                if (d <= bound) sr.push({d, key_of(j), j});
                continue;
              }
              const int64_t d = dist[v] + ((int64_t)iec[e].y << F) - pi[v] + pi[j];
              if (d <= bound && closed[j] != round && (reached[j] != round || d < dist[j])) {
                reached[j] = round; dist[j] = d; via[j] = e; pred[j] = v;
                sr.push({d, key_of(j), j});
                note(j, d);
              }
            }
          } else {
            // R_u: reverse arcs of saturated arcs x -> u (the twins of row u)
            const int32_t u = v - n;
            for (int32_t f = irp[u]; f < irp[u + 1]; ++f) {
              const int32_t a = twin[f];
              if (!y[a]) continue;
              const int32_t j = iec[f].x;  // L_x, the tail of arc a
              if (blocked && outside(j)) {
                const int64_t d = dist[v] - ((int64_t)iec[f].y << F) - pi[v] + pi0(j);
                if (d <= bound) sr.push({d, key_of(j), j});
                continue;
              }
              const int64_t d = dist[v] - ((int64_t)iec[f].y << F) - pi[v] + pi[j];
              if (d <= bound && closed[j] != round && (reached[j] != round || d < dist[j])) {
                reached[j] = round; dist[j] = d; via[j] = a; pred[j] = v;
                sr.push({d, key_of(j), j});
                note(j, d);
              }
            }
          }
        }
        if (t < 0) {
          if (blocked) break;  // dropped or nothing found: left to the next phase
          return 7;
        }
        for (int32_t j = t; j != s; j = pred[j]) y[via[j]] = (uint8_t)(j >= n);  // push one unit
        excess[s] -= 1;
        excess[t] += 1;
        ++pushes;
        const int64_t dt = dist[t];
        for (int32_t v : sr.order) pi[v] += dt - dist[v];
      }
    }
  }
  *pushes_out += pushes;
  return 0;
}

// runs items 0 .. count-1 on up to `threads` workers (dynamic hand-out)
template <typename Fn>
int run_items(int32_t count, int32_t threads, FinisherWork* w, std::vector<int64_t>& pushes, Fn fn) {
  int32_t nw = threads < 1 ? 1 : threads;
  if (nw > count) nw = count;
  if (nw < 1) return 0;
  if ((int32_t)w->workers.size() < nw) w->workers.resize(nw);
  if ((int32_t)pushes.size() < nw) pushes.resize(nw, 0);
  std::atomic<int32_t> next{0};
  std::atomic<int> status{0};
  auto run = [&](int32_t k) {
    for (;;) {
      const int32_t item = next.fetch_add(1);
      if (item >= count || status.load() != 0) break;
      const int r = fn(item, w->workers[k], &pushes[k]);
      if (r != 0) status.store(r);
    }
  };
  if (nw == 1) {
    run(0);
  } else {
    std::lock_guard<std::mutex> turn(g_pool_turn);
    worker_pool().run(nw, run);
  }
  return status.load();
}

}  // namespace

int host_finisher(int32_t n, const int32_t* irp, const int2* iec, const int32_t* twin, uint8_t* y,
                  const int32_t* exl, const int32_t* lam, int32_t F, int32_t* lam2,
                  const int32_t* seg_off, int32_t nseg, const uint8_t* include, int32_t threads,
                  int64_t* augmentations, FinisherWork* w, FinisherStats* stats, int64_t* ext_pi,
                  int32_t* ext_ex) {
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
  auto pushes_total = [](const std::vector<int64_t>& v) {
    int64_t t = 0;
    for (int64_t p : v) t += p;
    return t;
  };
  finisher_work_reserve(w, n);
  if (w->stamp.load() > (1u << 31)) {  // far from wrapping: clear the stamps and restart
    std::fill(w->reached.begin(), w->reached.end(), 0u);
    std::fill(w->closed.begin(), w->closed.end(), 0u);
    w->stamp.store(0);
    for (Searcher& sr : w->workers) sr.stamp_next = sr.stamp_end = 0;
  }
  // ext_pi / ext_ex: potentials and surpluses left by phase 1 run elsewhere
  // (the GPU); the host then starts at phase 2
  w->pi_p = ext_pi ? ext_pi : w->pi.data();
  w->ex_p = ext_ex ? ext_ex : w->excess.data();
  const bool skip1 = ext_pi && ext_ex;
  int64_t* pi = w->pi_p;
  int32_t* excess = w->ex_p;
  // phase 1: blocks of every segment, each first setting its own nodes'
  // potentials (lam, -lam) and surpluses; phase 2: larger blocks, from a copy
  // of the potentials phase 1 left; phase 3: whole segments
  std::vector<int2> blocks, blocks2;
  std::vector<int32_t> segs;
  for (int32_t sg = 0; sg < nseg; ++sg) {
    if (include && !include[sg]) continue;  // left alone: not read, not written
    segs.push_back(sg);
    for (int32_t b0 = seg_off[sg]; b0 < seg_off[sg + 1]; b0 += kFinBlock)
      blocks.push_back(make_int2(b0, std::min(b0 + kFinBlock, seg_off[sg + 1])));
    for (int32_t b0 = seg_off[sg]; b0 < seg_off[sg + 1]; b0 += kFinBlock2)
      blocks2.push_back(make_int2(b0, std::min(b0 + kFinBlock2, seg_off[sg + 1])));
  }
  std::vector<int64_t> pushes;
  auto t0 = clk::now();
  int r = skip1 ? 0 : run_items((int32_t)blocks.size(), threads, w, pushes,
                    [&](int32_t k, Searcher& sr, int64_t* p) {
                      for (int32_t i = blocks[k].x; i < blocks[k].y; ++i) {
                        pi[i] = lam[i];
                        pi[n + i] = -(int64_t)lam[i];
                        excess[i] = exl[i];       // L_i: supply b_i minus outflow
                        excess[n + i] = -exl[i];  // R_i: inflow minus demand b_i (z is symmetric)
                      }
                      return solve_range(n, blocks[k].x, blocks[k].y, lam, nullptr, irp, iec, twin, y, F, w,
                                         sr, p);
                    });
  int64_t done1 = pushes_total(pushes);
  if (stats && !skip1) {
    stats->ms_phase[0] += ms_since(t0);
    stats->aug[0] += done1;
    stats->threads = std::max<int32_t>(stats->threads, std::min<int32_t>(threads, (int32_t)blocks.size()));
  }
  t0 = clk::now();
  int64_t* pi_start = w->pi_start.data();
  if (r == 0)  // the potentials at phase 2's start, per block (every block copies its own nodes)
    r = run_items((int32_t)blocks2.size(), threads, w, pushes, [&](int32_t k, Searcher&, int64_t*) {
      const int32_t a = blocks2[k].x, b = blocks2[k].y;
      std::copy(pi + a, pi + b, pi_start + a);
      std::copy(pi + n + a, pi + n + b, pi_start + n + a);
      return 0;
    });
  if (r == 0)
    r = run_items((int32_t)blocks2.size(), threads, w, pushes,
                  [&](int32_t k, Searcher& sr, int64_t* p) {
                    return solve_range(n, blocks2[k].x, blocks2[k].y, nullptr, pi_start, irp, iec, twin, y, F,
                                       w, sr, p);
                  });
  const int64_t done2 = pushes_total(pushes);
  if (stats) {
    stats->ms_phase[1] += ms_since(t0);
    stats->aug[1] += done2 - done1;
  }
  t0 = clk::now();
  // phase 3: per segment, the plain search from each node still holding a
  // surplus (collected per phase-2 block, in key order)
  std::vector<std::vector<int32_t>> left(blocks2.size());
  if (r == 0)
    r = run_items((int32_t)blocks2.size(), threads, w, pushes, [&](int32_t k, Searcher&, int64_t*) {
      std::vector<int32_t>& out = left[k];
      out.clear();
      for (int32_t i = blocks2[k].x; i < blocks2[k].y; ++i) {
        if (excess[i] > 0) out.push_back(i);
        if (excess[n + i] > 0) out.push_back(n + i);
      }
      return 0;
    });
  std::vector<std::vector<int32_t>> seg_src(segs.size());
  for (size_t k = 0, q = 0; k < segs.size(); ++k) {
    const int32_t sg = segs[k];
    for (; q < blocks2.size() && blocks2[q].x < seg_off[sg + 1]; ++q)
      seg_src[k].insert(seg_src[k].end(), left[q].begin(), left[q].end());
  }
  if (r == 0)
    r = run_items((int32_t)segs.size(), threads, w, pushes, [&](int32_t k, Searcher& sr, int64_t* p) {
      const int32_t sg = segs[k];
      return solve_range(n, seg_off[sg], seg_off[sg + 1], nullptr, nullptr, irp, iec, twin, y, F, w, sr, p,
                         seg_src[k].data(), (int64_t)seg_src[k].size());
    });
  const int64_t total3 = pushes_total(pushes);
  if (r == 0)  // lambda at F + 1 bits: pi(L_i) - pi(R_i), block by block
    r = run_items((int32_t)blocks2.size(), threads, w, pushes, [&](int32_t k, Searcher&, int64_t*) {
      int st = 0;
      for (int32_t i = blocks2[k].x; i < blocks2[k].y; ++i) {
        const int64_t l2 = pi[i] - pi[n + i];
        if (l2 >= 2 * kLamLimit || l2 <= -2 * kLamLimit) st = 5;
        lam2[i] = (int32_t)l2;
      }
      return st;
    });
  const int64_t total = total3;
  if (stats) {
    stats->ms_phase[2] += ms_since(t0);
    stats->aug[2] += total - done2;
  }
  *augmentations = total;
  return r;
}

}  // namespace f2m
