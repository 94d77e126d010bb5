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

// Search state of one worker: heap, settled list and visit stamps.  Every
// push and pop writes the vectors' bounds, so each worker's state has cache
// lines of its own (128 bytes: adjacent-line prefetch pairs 64-byte lines).
struct alignas(128) Searcher {
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
// The phases of one finisher call follow each other closely, so a worker that
// finished a job, and the caller waiting for the workers, first poll for up to
// kSpinMicros before they sleep on the condition variable: a sleeping thread
// takes tens of microseconds to wake, which is the length of a whole phase.
constexpr int64_t kSpinMicros = 200;

struct WorkerPool {
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_job, cv_done;
  uint64_t generation = 0;               // bumped for every job (under mu)
  std::atomic<uint64_t> published{0};    // the same, for polling
  std::atomic<int32_t> busy{0};          // workers still on the current job
  std::atomic<bool> quit{false};
  uint64_t wake_seq = 0;             // bumped by wake() (under mu)
  std::function<void(int32_t)> job;  // runs as worker k (k >= 1)
  int32_t job_workers = 0;           // workers 1 .. job_workers - 1 take part

  // polls `done` for up to kSpinMicros; true if it became true
  template <typename Pred>
  static bool spin(Pred done) {
    const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(kSpinMicros);
    for (uint32_t it = 0;; ++it) {
      if (done()) return true;
      if ((it & 255u) == 255u && std::chrono::steady_clock::now() > until) return false;
    }
  }

  void start(int32_t nw) {  // nw - 1 threads (the caller is worker 0)
    for (int32_t k = (int32_t)threads.size() + 1; k < nw; ++k)
      threads.emplace_back([this, k] {
        uint64_t seen = 0, seen_wake = 0;
        for (;;) {
          spin([&] { return published.load(std::memory_order_acquire) != seen || quit.load(); });
          std::function<void(int32_t)> fn;
          {
            std::unique_lock<std::mutex> lk(mu);
            cv_job.wait(lk, [&] { return quit.load() || generation != seen || wake_seq != seen_wake; });
            if (quit.load()) return;
            seen_wake = wake_seq;
            if (generation == seen) continue;  // woken ahead of a job: poll for it
            seen = generation;
            if (k >= job_workers) continue;
            fn = job;
          }
          fn(k);
          if (busy.fetch_sub(1, std::memory_order_acq_rel) == 1) {
            std::lock_guard<std::mutex> lk(mu);
            cv_done.notify_all();
          }
        }
      });
  }
  // wakes the workers 1 .. nw - 1 (creating them if needed) to poll for a
  // job that is about to come
  void wake(int32_t nw) {
    start(nw);
    {
      std::lock_guard<std::mutex> lk(mu);
      ++wake_seq;
    }
    cv_job.notify_all();
  }
  void run(int32_t nw, const std::function<void(int32_t)>& fn) {
    start(nw);
    {
      std::lock_guard<std::mutex> lk(mu);
      job = fn;
      job_workers = nw;
      busy.store(nw - 1);
      ++generation;
      published.store(generation, std::memory_order_release);
    }
    cv_job.notify_all();
    fn(0);
    if (!spin([&] { return busy.load(std::memory_order_acquire) == 0; })) {
      std::unique_lock<std::mutex> lk(mu);
      cv_done.wait(lk, [&] { return busy.load(std::memory_order_acquire) == 0; });
    }
    std::lock_guard<std::mutex> lk(mu);
    job = nullptr;
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(mu);
      quit.store(true);
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

void finisher_pool_wake(int32_t threads) {
  if (threads < 2) return;
  std::unique_lock<std::mutex> turn(g_pool_turn, std::try_to_lock);
  if (turn.owns_lock()) worker_pool().wake(threads);  // (busy with another job: nothing to do)
}

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
// key order -- the others are skipped without a look.  settled (optional)
// collects the nodes whose potential an augmentation raised.
int solve_range(int32_t n, int32_t lo, int32_t hi, const int32_t* lam0, const int64_t* pi0v,
                const int32_t* irp, const int2* iec, const int32_t* twin, uint8_t* y, int32_t F,
                FinisherWork* w, Searcher& sr, int64_t* pushes_out, const int32_t* srcs = nullptr,
                int64_t nsrc = 0, std::vector<int32_t>* settled = nullptr) {
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
        if (settled) settled->insert(settled->end(), sr.order.begin(), sr.order.end());
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
  int64_t* pi_start = w->pi_start.data();
  // lambda at F + 1 bits, pi(L_i) - pi(R_i): every block writes it for its
  // nodes when it is done, and the later phases again for the nodes they
  // settle (no other potential changes); a value out of range is noted, and
  // the range is then checked on the final values
  std::atomic<bool> any_wide{false};
  auto write_lam2 = [&](int32_t i) {
    const int64_t l2 = pi[i] - pi[n + i];
    lam2[i] = (int32_t)l2;
    return l2 >= 2 * kLamLimit || l2 <= -2 * kLamLimit;
  };
  auto write_lam2_nodes = [&](const std::vector<int32_t>& nodes) {  // L or R copies
    bool wd = false;
    for (int32_t v : nodes) wd |= write_lam2(v < n ? v : v - n);
    if (wd) any_wide.store(true);
  };
  // a block's nodes still holding a surplus, in key order
  auto sources_left = [&](int32_t a, int32_t b, std::vector<int32_t>& out) {
    out.clear();
    for (int32_t i = a; i < b; ++i) {
      if (excess[i] > 0) out.push_back(i);
      if (excess[n + i] > 0) out.push_back(n + i);
    }
  };
  // phase 1 from each block's sources; every block then copies its nodes'
  // potentials into pi_start (phase 1 writes no other node's, so that is the
  // state phase 2 starts from), writes their lambda and keeps the sources it
  // left for phase 2
  std::vector<std::vector<int32_t>> left1(skip1 ? 0 : blocks.size());
  auto t0 = clk::now();
  int r = skip1 ? 0 : run_items((int32_t)blocks.size(), threads, w, pushes,
                    [&](int32_t k, Searcher& sr, int64_t* p) {
                      const int32_t a = blocks[k].x, b = blocks[k].y;
                      std::vector<int32_t>& src = left1[k];  // the block's sources, in key order
                      src.clear();
                      for (int32_t i = a; i < b; ++i) {
                        pi[i] = lam[i];
                        pi[n + i] = -(int64_t)lam[i];
                        excess[i] = exl[i];       // L_i: supply b_i minus outflow
                        excess[n + i] = -exl[i];  // R_i: inflow minus demand b_i (z is symmetric)
                        if (exl[i] > 0) src.push_back(i);
                        if (exl[i] < 0) src.push_back(n + i);
                      }
                      const int rc = solve_range(n, a, b, lam, nullptr, irp, iec, twin, y, F, w, sr, p,
                                                 src.data(), (int64_t)src.size());
                      std::copy(pi + a, pi + b, pi_start + a);
                      std::copy(pi + n + a, pi + n + b, pi_start + n + a);
                      bool wd = false;
                      for (int32_t i = a; i < b; ++i) wd |= write_lam2(i);
                      if (wd) any_wide.store(true);
                      size_t kept = 0;  // a surplus never grows: the sources left are among these
                      for (int32_t v : src)
                        if (excess[v] > 0) src[kept++] = v;
                      src.resize(kept);
                      return rc;
                    });
  int64_t done1 = pushes_total(pushes);
  if (stats && !skip1) {
    stats->ms_phase[0] += ms_since(t0);
    stats->aug[0] += done1;
    stats->threads = std::max<int32_t>(stats->threads, std::min<int32_t>(threads, (int32_t)blocks.size()));
  }
  t0 = clk::now();
  if (r == 0 && skip1)  // phase 1 ran elsewhere: the copy is taken here
    r = run_items((int32_t)blocks2.size(), threads, w, pushes, [&](int32_t k, Searcher&, int64_t*) {
      const int32_t a = blocks2[k].x, b = blocks2[k].y;
      std::copy(pi + a, pi + b, pi_start + a);
      std::copy(pi + n + a, pi + n + b, pi_start + n + a);
      return 0;
    });
  // phase 2, from the sources phase 1 left (a phase-2 block is a run of
  // whole phase-1 blocks: both start at the segment's first node, and
  // kFinBlock2 is a multiple of kFinBlock); each block then lists its sources
  // left for phase 3 and writes lambda for the nodes it settled
  static_assert(kFinBlock2 % kFinBlock == 0, "phase-2 blocks are runs of phase-1 blocks");
  std::vector<int32_t> first1(blocks2.size() + 1, 0);  // phase-1 blocks of phase-2 block k
  if (!skip1) {
    size_t q = 0;
    for (size_t k = 0; k < blocks2.size(); ++k) {
      while (q < blocks.size() && blocks[q].x < blocks2[k].x) ++q;
      first1[k] = (int32_t)q;
    }
    first1[blocks2.size()] = (int32_t)blocks.size();
  }
  std::vector<std::vector<int32_t>> left(blocks2.size()), src2(blocks2.size()), settled2(blocks2.size());
  if (r == 0)
    r = run_items((int32_t)blocks2.size(), threads, w, pushes,
                  [&](int32_t k, Searcher& sr, int64_t* p) {
                    const int32_t a = blocks2[k].x, b = blocks2[k].y;
                    if (skip1) {  // no lists from phase 1: every node is a candidate
                      const int rc = solve_range(n, a, b, nullptr, pi_start, irp, iec, twin, y, F, w, sr, p);
                      sources_left(a, b, left[k]);
                      bool wd = false;
                      for (int32_t i = a; i < b; ++i) wd |= write_lam2(i);
                      if (wd) any_wide.store(true);
                      return rc;
                    }
                    std::vector<int32_t>& src = src2[k];
                    src.clear();
                    for (int32_t q = first1[k]; q < first1[k + 1]; ++q)
                      src.insert(src.end(), left1[q].begin(), left1[q].end());
                    settled2[k].clear();
                    const int rc = solve_range(n, a, b, nullptr, pi_start, irp, iec, twin, y, F, w, sr, p,
                                               src.data(), (int64_t)src.size(), &settled2[k]);
                    left[k].clear();  // a surplus never grows: the sources left are among these
                    for (int32_t v : src)
                      if (excess[v] > 0) left[k].push_back(v);
                    write_lam2_nodes(settled2[k]);
                    return rc;
                  });
  const int64_t done2 = pushes_total(pushes);
  if (stats) {
    stats->ms_phase[1] += ms_since(t0);
    stats->aug[1] += done2 - done1;
  }
  t0 = clk::now();
  // phase 3: per segment, the plain search from each node still holding a
  // surplus
  std::vector<std::vector<int32_t>> seg_src(segs.size()), settled(segs.size());
  for (size_t k = 0, q = 0; k < segs.size(); ++k) {
    const int32_t sg = segs[k];
    for (; q < blocks2.size() && blocks2[q].x < seg_off[sg + 1]; ++q)
      seg_src[k].insert(seg_src[k].end(), left[q].begin(), left[q].end());
  }
  if (r == 0)
    r = run_items((int32_t)segs.size(), threads, w, pushes, [&](int32_t k, Searcher& sr, int64_t* p) {
      const int32_t sg = segs[k];
      settled[k].clear();
      const int rc = solve_range(n, seg_off[sg], seg_off[sg + 1], nullptr, nullptr, irp, iec, twin, y, F, w, sr,
                                 p, seg_src[k].data(), (int64_t)seg_src[k].size(), &settled[k]);
      write_lam2_nodes(settled[k]);
      return rc;
    });
  const int64_t total3 = pushes_total(pushes);
  if (r == 0 && any_wide.load()) {  // some lambda was out of range on the way: check the final values
    bool wd = false;
    for (const int2& bl : blocks2)
      for (int32_t i = bl.x; i < bl.y; ++i) wd |= write_lam2(i);
    if (wd) r = 5;
  }
  const int64_t total = total3;
  if (stats) {
    stats->ms_phase[2] += ms_since(t0);
    stats->aug[2] += total - done2;
  }
  *augmentations = total;
  return r;
}

}  // namespace f2m
