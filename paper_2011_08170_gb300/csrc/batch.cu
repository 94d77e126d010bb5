// Batched solve: many independent F2M instances in one context.
//
// The instances become one disjoint union of segments (instance s = nodes
// [seg_off[s], seg_off[s+1]) of the union).  Every device step of a solve
// covers all instances at once -- one persistent GDP launch per phase
// (gdp_batch_kernel, converged instances frozen), one pricing scan over the
// tile pairs of the instances that need one, one merge, one extraction, one
// finisher call -- and the host keeps, per instance, the state of the solve
// loop of f2m_solve.  Since no step mixes instances, each instance's lambda,
// x and bound are those of its own solve (the finisher is told which
// instances it may touch).
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <chrono>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/f2m.h"
#include "ctx_internal.h"
#include "f2m_internal.h"

using namespace f2m;

struct f2m_batch {
  f2m_ctx* u = nullptr;            // the union context
  int32_t count = 0;
  std::vector<int32_t> n;          // nodes per instance
  // device scratch of the batch GDP phase
  uint8_t* d_active = nullptr;
  unsigned long long* d_seg_ch = nullptr;
  long long* d_seg_sweeps = nullptr;
  // tiles of the chosen kernel shape over the current CSR, all instances (host)
  std::vector<int4> tiles_all;
  std::vector<int32_t> e1_all;
  int32_t shape = -1;               // batch kernel shape in use
  int32_t grid = 0;
  int64_t tiles_version = -1;
  // the list of one launch: pinned host copy -> device (captured launch reads them)
  int4* h_tiles = nullptr;
  int32_t* h_e1 = nullptr;
  BatchChunk* h_chunk = nullptr;
  int4* d_tiles = nullptr;
  int32_t* d_e1 = nullptr;
  BatchChunk* d_chunk = nullptr;
  int32_t tiles_cap = 0;
  // captured launch (list upload, resets, kernel, read-backs), replayed on a private stream
  cudaStream_t gs = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_version = -1;       // tiles_version the graph belongs to
  long long graph_kernels = 0;      // kernels per replay
  bool graph_failed = false;
  cudaEvent_t e_in = nullptr, e_out = nullptr;
  uint8_t* h_active = nullptr;      // pinned copies read / written by the phase
  GdpCtl* h_ctl = nullptr;
  long long* h_sw = nullptr;
  uint8_t* h_still = nullptr;
  long long* d_seg_b2 = nullptr;
  unsigned long long* d_seg_bad = nullptr;
  int32_t* d_tmp_a = nullptr;       // output staging
  int32_t* d_tmp_b = nullptr;
  int64_t tmp_cap = 0;
  uint8_t* d_mask = nullptr;        // per-segment mask for the masked steps
  // results, snapshotted when an instance finishes (later steps for other
  // instances move entries and rescale lambda)
  int32_t* d_res_lam = nullptr;     // [N] lambda, units 2^-res_fb[s]
  int32_t* d_res_rp = nullptr;      // [N + count] local row offsets per instance
  int2* d_res_ec = nullptr;         // arena of {col (union id), cost}
  uint8_t* d_res_x2 = nullptr;      // arena of x in half units
  int64_t res_cap = 0, res_used = 0;
  int32_t* h_irp = nullptr;         // pinned copy of the internal row offsets (tile packing)
  int32_t tiles_te = -1, tiles_tn = -1;  // tile limits tiles_all was packed with
  long long* h_snap = nullptr;      // pinned staging of a snapshot
  long long* d_snap_eoff = nullptr; // [count] arena offset of each instance being copied
  uint8_t* d_snap_done = nullptr;   // [count] instances being copied
  int32_t* d_snap_ent = nullptr;    // [count + 1] first entry of each instance
  std::vector<int64_t> res_eoff, res_nnz, res_b2;
  std::vector<int32_t> res_fb;
  std::vector<uint8_t> res_done;
  // cluster path (gdp_cluster.cu): one thread-block cluster per instance
  struct ClusterClass {
    int32_t C = 0, threads = 0, emax = 0, nmax = 0;
  };
  bool used_clusters = false;       // the last phase ran on clusters
  int64_t cl_version = -1;          // GdpPlan::version the cluster plan belongs to
  bool cl_ok = false;               // every instance fits a cluster that fits the device
  std::vector<int32_t> cl_class_of; // class (0..4: C = 1, 2, 4, 8, 16) per instance
  std::vector<ClusterInst> cl_inst; // per instance
  ClusterClass cl_cls[5];
  int2* d_pk = nullptr;             // packed rows of every instance
  int64_t pk_cap = 0;
  ClusterInst* d_cl_all = nullptr;  // all instances (packing)
  ClusterInst* d_cl_list = nullptr; // a phase's lists, class by class
  ClusterInst* h_cl_list = nullptr;
  ClusterOut* d_cl_out = nullptr;
  ClusterOut* h_cl_out = nullptr;
  cudaStream_t cl_st[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t cl_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace {

f2m_status bfail(f2m_batch* b, f2m_status s, const std::string& msg) {
  return fail(b ? b->u : nullptr, s, msg);
}

}  // namespace

extern "C" void f2m_destroy_batch(f2m_batch* b) {
  if (!b) return;
  DevSyncedScope synced;  // one wait for the device, then every block goes to the cache
  if (b->u) f2m_destroy(b->u);
  dfree(b->d_active); dfree(b->d_seg_ch); dfree(b->d_seg_sweeps); dfree(b->d_tiles); dfree(b->d_e1);
  dfree(b->d_snap_eoff); dfree(b->d_snap_done); dfree(b->d_snap_ent);
  if (b->h_snap) cudaFreeHost(b->h_snap);
  if (b->h_irp) cudaFreeHost(b->h_irp);
  dfree(b->d_chunk);
  if (b->h_tiles) cudaFreeHost(b->h_tiles);
  if (b->h_e1) cudaFreeHost(b->h_e1);
  if (b->h_chunk) cudaFreeHost(b->h_chunk);
  dfree(b->d_seg_b2); dfree(b->d_seg_bad); dfree(b->d_tmp_a); dfree(b->d_tmp_b);
  dfree(b->d_mask); dfree(b->d_res_lam); dfree(b->d_res_rp); dfree(b->d_res_ec); dfree(b->d_res_x2);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->gs) cudaStreamDestroy(b->gs);
  if (b->e_in) cudaEventDestroy(b->e_in);
  if (b->e_out) cudaEventDestroy(b->e_out);
  if (b->h_active) cudaFreeHost(b->h_active);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->h_sw) cudaFreeHost(b->h_sw);
  if (b->h_still) cudaFreeHost(b->h_still);
  dfree(b->d_pk); dfree(b->d_cl_all); dfree(b->d_cl_list); dfree(b->d_cl_out);
  if (b->h_cl_list) cudaFreeHost(b->h_cl_list);
  if (b->h_cl_out) cudaFreeHost(b->h_cl_out);
  for (cudaStream_t& q : b->cl_st)
    if (q) cudaStreamDestroy(q);
  for (cudaEvent_t& q : b->cl_ev)
    if (q) cudaEventDestroy(q);
  delete b;
}

extern "C" f2m_status f2m_create_batch(int32_t count, const int32_t* n, const int32_t* xy,
                                       const int32_t* row_ptr, const int32_t* col,
                                       const f2m_params* params, void* stream, f2m_batch** out) {
  if (!out) return fail(nullptr, F2M_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !n || !xy || !row_ptr || !col)
    return fail(nullptr, F2M_ERR_INVALID_ARG, "count < 1 or NULL array");
  std::vector<int32_t> seg_off(count + 1, 0);
  for (int32_t s = 0; s < count; ++s) {
    if (n[s] < 4) return fail(nullptr, F2M_ERR_INVALID_ARG, "instance " + std::to_string(s) + ": n < 4");
    if ((int64_t)seg_off[s] + n[s] >= (1 << 24))
      return fail(nullptr, F2M_ERR_INVALID_ARG, "total nodes must stay below 2^24");
    seg_off[s + 1] = seg_off[s] + n[s];
  }
  const int32_t N = seg_off[count];
  cudaStream_t st = (cudaStream_t)stream;
  // per-instance entry counts: the last offset of each local row_ptr
  std::vector<int32_t> eoff(count + 1, 0);
  {
    std::vector<int32_t> rp_all(N + count);
    cudaError_t e = cudaMemcpyAsync(rp_all.data(), row_ptr, sizeof(int32_t) * (N + count),
                                    cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "create_batch: read row_ptr");
    for (int32_t s = 0; s < count; ++s) {
      const int64_t nz = rp_all[seg_off[s + 1] + s];
      if (nz < 0 || (int64_t)eoff[s] + nz >= INT32_MAX)
        return fail(nullptr, F2M_ERR_INVALID_ARG, "instance " + std::to_string(s) + ": bad row_ptr");
      eoff[s + 1] = eoff[s] + (int32_t)nz;
    }
  }
  const int64_t nnz = eoff[count];
  // union CSR on the device
  int32_t *d_rpl = nullptr, *d_coll = nullptr, *d_rp = nullptr, *d_col = nullptr, *d_so = nullptr,
          *d_eo = nullptr;
  CheckCtl* d_chk = nullptr;
  f2m_status s = F2M_OK;
  do {
    cudaError_t e = dalloc(&d_rpl, N + count);
    if (e == cudaSuccess) e = dalloc(&d_coll, nnz);
    if (e == cudaSuccess) e = dalloc(&d_rp, N + 1);
    if (e == cudaSuccess) e = dalloc(&d_col, nnz);
    if (e == cudaSuccess) e = dalloc(&d_so, count + 1);
    if (e == cudaSuccess) e = dalloc(&d_eo, count + 1);
    if (e == cudaSuccess) e = dalloc(&d_chk, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rpl, row_ptr, sizeof(int32_t) * (N + count), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_coll, col, sizeof(int32_t) * nnz, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_so, seg_off.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_eo, eoff.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, st);
    CheckCtl h0{0, INT32_MAX};
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_chk, &h0, sizeof(h0), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_batch_union(d_rpl, d_coll, d_so, d_eo, count, N, nnz, d_rp, d_col, d_chk, st);
    CheckCtl h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_chk, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { s = cuda_fail(nullptr, e, "create_batch: union"); break; }
    if (h.flags) {
      s = fail(nullptr, F2M_ERR_INVALID_ARG,
               std::string(h.flags & 2 ? "column index outside its instance" : "row_ptr out of range") +
                   " (at " + std::to_string(h.first_bad) + ")");
      break;
    }
    f2m_ctx* u = nullptr;
    s = create_internal(xy, N, d_rp, d_col, params, stream, seg_off, &u);
    if (s != F2M_OK) break;
    f2m_batch* b = new (std::nothrow) f2m_batch();
    if (!b) { f2m_destroy(u); s = fail(nullptr, F2M_ERR_OOM, "host allocation"); break; }
    b->u = u;
    b->count = count;
    b->n.assign(n, n + count);
    e = dalloc(&u->d_seg_off, count + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u->d_seg_off, seg_off.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = dalloc(&b->d_active, count);
    if (e == cudaSuccess) e = dalloc(&b->d_seg_ch, 3LL * count);
    if (e == cudaSuccess) e = dalloc(&b->d_seg_sweeps, count);
    if (e == cudaSuccess) e = dalloc(&b->d_seg_b2, count);
    if (e == cudaSuccess) e = dalloc(&b->d_seg_bad, count);
    if (e == cudaSuccess) e = dalloc(&u->d_fin_include, count);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->d_fin_include, 1, count, st);
    if (e == cudaSuccess) e = dalloc(&b->d_mask, count);
    if (e == cudaSuccess) e = dalloc(&b->d_res_lam, N);
    if (e == cudaSuccess) e = dalloc(&b->d_res_rp, (int64_t)N + count);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->e_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->e_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_active, count);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ctl, sizeof(GdpCtl));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_sw, sizeof(long long) * count);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_still, count);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_chunk, sizeof(BatchChunk));
    if (e == cudaSuccess) e = dalloc(&b->d_chunk, 1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { f2m_destroy_batch(b); s = cuda_fail(nullptr, e, "create_batch: setup"); break; }
    *out = b;
  } while (0);
  dfree(d_rpl); dfree(d_coll); dfree(d_rp); dfree(d_col); dfree(d_so); dfree(d_eo); dfree(d_chk);
  return s;
}

// ---- GDP phase: tiles, kernel shape (autotuned), captured launch ----------------------

// tiles of at most te entries and tn nodes over the current renumbered CSR
// (host lists: {first node, end node, instance, first entry} and end entries)
static f2m_status batch_tiles(f2m_batch* b, int te, int tn, std::vector<int4>& tiles, std::vector<int32_t>& e1) {
  f2m_ctx* c = b->u;
  GdpPlan& P = c->plan;
  if (!b->h_irp) CK(c, cudaMallocHost((void**)&b->h_irp, sizeof(int32_t) * (c->n + 1)));
  const int32_t* irp = b->h_irp;
  CK(c, cudaMemcpyAsync(b->h_irp, P.irp, sizeof(int32_t) * (c->n + 1), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  // pack the node range [v, end) of segment s greedily: at most tn nodes and te entries a tile
  auto pack = [&](int32_t s, int32_t v, int32_t end, std::vector<int4>& t_out, std::vector<int32_t>& e_out) {
    while (v < end) {
      const int32_t start = v, e0 = irp[v];
      while (v < end && v - start < tn && irp[v + 1] - e0 <= te) ++v;
      if (v == start) return false;
      t_out.push_back(make_int4(start, v, s, e0));
      e_out.push_back(irp[v]);
    }
    return true;
  };
  const bool own = &tiles == &b->tiles_all;  // the phase's list (the autotuner packs its own)
  const bool update = own && b->tiles_te == te && b->tiles_tn == tn && !tiles.empty();
  std::vector<int4> nt;
  std::vector<int32_t> ne;
  nt.reserve(tiles.size() + 64);
  ne.reserve(tiles.size() + 64);
  if (update) {
    // a merge only adds entries: keep every tile's node range with its new
    // entry range, and pack again only a range that now holds too many entries
    for (const int4& t : tiles) {
      const int32_t e0 = irp[t.x], e1v = irp[t.y];
      if (e1v - e0 <= te) {
        nt.push_back(make_int4(t.x, t.y, t.z, e0));
        ne.push_back(e1v);
      } else if (!pack(t.z, t.x, t.y, nt, ne)) {
        return fail(c, F2M_ERR_INVALID_ARG, "a node has more candidate edges than a batch tile holds");
      }
    }
  } else {
    for (int32_t s = 0; s < b->count; ++s)
      if (!pack(s, c->seg_off[s], c->seg_off[s + 1], nt, ne))
        return fail(c, F2M_ERR_INVALID_ARG, "a node has more candidate edges than a batch tile holds");
  }
  tiles.swap(nt);
  e1.swap(ne);
  if (own) {
    b->tiles_te = te;
    b->tiles_tn = tn;
  }
  return F2M_OK;
}

// room for `need` tiles in the pinned and device list buffers (drops the captured graph)
static f2m_status batch_list_reserve(f2m_batch* b, int32_t need) {
  f2m_ctx* c = b->u;
  if (need <= b->tiles_cap) return F2M_OK;
  CK(c, cudaStreamSynchronize(c->st));
  CK(c, cudaStreamSynchronize(b->gs));
  if (b->h_tiles) cudaFreeHost(b->h_tiles);
  if (b->h_e1) cudaFreeHost(b->h_e1);
  b->h_tiles = nullptr;
  b->h_e1 = nullptr;
  dfree(b->d_tiles);
  dfree(b->d_e1);
  b->tiles_cap = 0;
  const int32_t cap = need + need / 8 + 64;
  CK(c, cudaMallocHost((void**)&b->h_tiles, sizeof(int4) * cap));
  CK(c, cudaMallocHost((void**)&b->h_e1, sizeof(int32_t) * cap));
  CK(c, dalloc(&b->d_tiles, cap));
  CK(c, dalloc(&b->d_e1, cap));
  b->tiles_cap = cap;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  return F2M_OK;
}

// CTAs of a cooperative launch of `shape` over up to ntiles tiles (0: the shape does not run)
static int32_t batch_grid(f2m_batch* b, int shape, int32_t ntiles) {
  const int sms = b->u->num_sms;
  int per_sm = batch_shape_blocks(shape, 1);
  const int32_t units = batch_shape_units(shape);
  for (int it = 0; it < 4 && per_sm > 0; ++it) {  // the tile table grows as the grid shrinks
    const int32_t G = sms * per_sm;
    const int32_t mcap = (int32_t)((ntiles + (int64_t)G * units - 1) / ((int64_t)G * units));
    const int p2 = batch_shape_blocks(shape, mcap);
    if (p2 >= per_sm) break;
    per_sm = p2;
  }
  if (per_sm < 1) return 0;
  int32_t G = sms * per_sm;
  if ((int64_t)G * units > ntiles) G = (int32_t)((ntiles + units - 1) / units);
  return G < 1 ? 1 : G;
}

// One launch on stream st: the list and parameters (pinned host -> device),
// per-launch resets, the persistent kernel, the results back to pinned memory.
static cudaError_t enqueue_launch(f2m_batch* b, cudaStream_t st, int shape, int32_t G, int32_t max_tiles) {
  f2m_ctx* c = b->u;
  GdpPlan& P = c->plan;
  cudaError_t e = cudaMemcpyAsync(b->d_chunk, b->h_chunk, sizeof(BatchChunk), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tiles, b->h_tiles, sizeof(int4) * b->tiles_cap, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_e1, b->h_e1, sizeof(int32_t) * b->tiles_cap, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_seg_ch, 0, sizeof(unsigned long long) * 3 * b->count, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_gdp, 0, sizeof(GdpCtl), st);
  if (e == cudaSuccess)
    e = launch_gdp_batch(shape, P.irp, P.iec, b->d_tiles, b->d_e1, b->d_chunk, max_tiles, G, b->count,
                         b->d_active, b->d_seg_ch, b->d_seg_sweeps, P.ilam[0], P.ilam[1], c->p.frac_bits,
                         c->p.damping_shift, c->d_gdp, c->p.barrier_budget_cycles, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_ctl, c->d_gdp, sizeof(GdpCtl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_sw, b->d_seg_sweeps, sizeof(long long) * b->count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_still, b->d_active, b->count, cudaMemcpyDeviceToHost, st);
  return e;
}

// start of a phase: lambda into the renumbered double buffer, active flags, sweep records
static cudaError_t enqueue_phase_start(f2m_batch* b, cudaStream_t st, const uint8_t* h_active) {
  f2m_ctx* c = b->u;
  GdpPlan& P = c->plan;
  cudaError_t e = gather_perm(c->d_lam[c->cur], P.perm, c->n, P.ilam[0], st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P.ilam[1], P.ilam[0], sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    if (h_active)
      e = cudaMemcpyAsync(b->d_active, h_active, b->count, cudaMemcpyHostToDevice, st);
    else
      e = cudaMemsetAsync(b->d_active, 1, b->count, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_seg_sweeps, 0, sizeof(long long) * b->count, st);
  return e;
}

// the list of one launch: the tiles of the instances flagged in `act`
static int32_t fill_list(f2m_batch* b, const std::vector<int4>& tiles, const std::vector<int32_t>& e1,
                         const uint8_t* act) {
  int32_t m = 0;
  for (size_t k = 0; k < tiles.size(); ++k) {
    if (act && !act[tiles[k].z]) continue;
    b->h_tiles[m] = tiles[k];
    b->h_e1[m] = e1[k];
    ++m;
  }
  return m;
}

// Process-wide choice of the autotuner, keyed by (SMs, instances, nodes,
// entries / 2^16): a batch of the same shape created again skips the trials.
static std::mutex g_tune_mu;
static std::map<std::array<long long, 4>, int> g_tune;

// Autotuner: time a few sweeps of every shape that runs on this batch (from
// the current lambda, all instances active, nothing kept) and keep the
// fastest per sweep.
static f2m_status batch_autotune(f2m_batch* b) {
  f2m_ctx* c = b->u;
  const std::array<long long, 4> key = {c->num_sms, b->count, c->n, c->nnz >> 16};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      b->shape = it->second;
      return F2M_OK;
    }
  }
  int best = -1;
  double best_t = 0;
  std::vector<int4> tiles;
  std::vector<int32_t> e1;
  for (int sh = 0; sh < batch_num_shapes(); ++sh) {
    int te = 0, tn = 0;
    batch_shape_tile(sh, &te, &tn);
    f2m_status s = batch_tiles(b, te, tn, tiles, e1);
    if (s != F2M_OK) return s;
    const int32_t nt = (int32_t)tiles.size();
    const int32_t G = batch_grid(b, sh, nt);
    if (G < 1) continue;
    s = batch_list_reserve(b, nt);
    if (s != F2M_OK) return s;
    fill_list(b, tiles, e1, nullptr);
    double t = 0;
    for (int rep = 0; rep < 2; ++rep) {  // the first run only warms up
      *b->h_chunk = BatchChunk{nt, 0, 0, rep == 0 ? 4 : 48};
      CK(c, enqueue_phase_start(b, c->st, nullptr));
      CK(c, cudaEventRecord(c->ev0, c->st));
      CK(c, enqueue_launch(b, c->st, sh, G, nt));
      CK(c, cudaEventRecord(c->ev1, c->st));
      CK(c, cudaStreamSynchronize(c->st));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev0, c->ev1);
      if (b->h_ctl->status & kGdpTimeout) return fail(c, F2M_ERR_TIMEOUT, "device-wide barrier wait exceeded its budget");
      t = ms / (double)(b->h_ctl->sweeps > 0 ? b->h_ctl->sweeps : 1);
    }
    if (best < 0 || t < best_t) {
      best = sh;
      best_t = t;
    }
  }
  if (best < 0) return fail(c, F2M_ERR_CUDA, "no batch kernel shape fits this device");
  b->shape = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return F2M_OK;
}

// Sweeps per launch of a phase: after each launch the list is rebuilt from the
// instances still active (even, so that every launch starts from buffer 0).
constexpr long long kSweepsPerLaunch = 256;

// One GDP phase over the instances flagged in `active` (host, one byte each);
// adds each instance's sweeps to sweeps_out.
// Cluster plan for the current graph: the cluster size of every instance
// (the smallest of 1, 2, 4, 8, 16 CTAs whose node and entry shares fit one
// CTA's shared memory), the per-class launch shape, and the packed rows.
static f2m_status cluster_plan(f2m_batch* b) {
  f2m_ctx* c = b->u;
  GdpPlan& P = c->plan;
  const int32_t K = b->count;
  b->cl_ok = false;
  b->cl_version = P.version;
  std::vector<int32_t> irp(c->n + 1);
  CK(c, cudaMemcpyAsync(irp.data(), P.irp, sizeof(int32_t) * (c->n + 1), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  b->cl_class_of.assign(K, -1);
  b->cl_inst.resize(K);
  for (auto& q : b->cl_cls) q = f2m_batch::ClusterClass{};
  for (int32_t s = 0; s < K; ++s) {
    const int32_t node0 = c->seg_off[s], n = c->seg_off[s + 1] - node0;
    for (int k = 0; k < 5; ++k) {
      const int32_t C = 1 << k, per = (n + C - 1) / C;
      if (per > kClusterNodes) continue;
      int32_t emax = 0;
      for (int32_t r = 0; r < C; ++r) {
        const int32_t a = std::min(node0 + r * per, node0 + n), e = std::min(a + per, node0 + n);
        emax = std::max(emax, irp[e] - irp[a]);
      }
      if (emax > kClusterEntries) continue;
      b->cl_class_of[s] = k;
      b->cl_inst[s] = ClusterInst{node0, n, per, s};
      auto& q = b->cl_cls[k];
      q.C = C;
      q.emax = std::max(q.emax, emax);
      q.nmax = std::max(q.nmax, per);
      break;
    }
    if (b->cl_class_of[s] < 0) return F2M_OK;  // too large: the streaming kernels
  }
  for (auto& q : b->cl_cls) {
    if (q.C == 0) continue;
    q.threads = std::min(1024, std::max(128, (q.nmax + 31) / 32 * 32));
    if (cluster_max_smem_ok(q.C, q.threads, q.emax, q.nmax) < 1) return F2M_OK;
  }
  if (!b->d_cl_all) {
    CK(c, dalloc(&b->d_cl_all, K));
    CK(c, dalloc(&b->d_cl_list, K));
    CK(c, dalloc(&b->d_cl_out, K));
    CK(c, cudaMallocHost((void**)&b->h_cl_list, sizeof(ClusterInst) * K));
    CK(c, cudaMallocHost((void**)&b->h_cl_out, sizeof(ClusterOut) * K));
    for (cudaStream_t& q : b->cl_st) CK(c, cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    for (cudaEvent_t& q : b->cl_ev) CK(c, cudaEventCreateWithFlags(&q, cudaEventDisableTiming));
  }
  if (b->pk_cap < c->nnz) {
    dfree(b->d_pk);
    b->pk_cap = c->ec_cap;
    CK(c, dalloc(&b->d_pk, b->pk_cap));
  }
  CK(c, cudaMemcpyAsync(b->d_cl_all, b->cl_inst.data(), sizeof(ClusterInst) * K, cudaMemcpyHostToDevice, c->st));
  CK(c, cluster_pack(P.irp, P.iec, b->d_cl_all, K, c->p.frac_bits, b->d_pk, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  b->cl_ok = true;
  return F2M_OK;
}

// A GDP phase with one cluster per active instance: the classes run side by
// side on their own streams; every instance stops at its own fixed point or
// after max_iters sweeps.
static f2m_status batch_cluster_phase(f2m_batch* b, const std::vector<uint8_t>& active,
                                      std::vector<int64_t>& sweeps_out, double* ms) {
  f2m_ctx* c = b->u;
  c->lam_version += 1;
  GdpPlan& P = c->plan;
  const int32_t K = b->count;
  CK(c, enqueue_phase_start(b, c->st, nullptr));
  CK(c, cudaMemsetAsync(b->d_cl_out, 0, sizeof(ClusterOut) * K, c->st));
  // lists of the active instances per class, larger instances first
  int32_t off[6] = {0, 0, 0, 0, 0, 0};
  int32_t m = 0;
  for (int k = 0; k < 5; ++k) {
    off[k] = m;
    const int32_t m0 = m;
    for (int32_t s = 0; s < K; ++s)
      if (active[s] && b->cl_class_of[s] == k) b->h_cl_list[m++] = b->cl_inst[s];
    std::sort(b->h_cl_list + m0, b->h_cl_list + m,
              [](const ClusterInst& x, const ClusterInst& y) { return x.n > y.n || (x.n == y.n && x.seg < y.seg); });
  }
  off[5] = m;
  if (m > 0) CK(c, cudaMemcpyAsync(b->d_cl_list, b->h_cl_list, sizeof(ClusterInst) * m, cudaMemcpyHostToDevice, c->st));
  CK(c, cudaEventRecord(c->ev0, c->st));
  CK(c, cudaEventRecord(b->cl_ev[5], c->st));
  for (int k = 4; k >= 0; --k) {  // the largest clusters first
    const int32_t cnt = off[k + 1] - off[k];
    if (cnt == 0) continue;
    const auto& q = b->cl_cls[k];
    CK(c, cudaStreamWaitEvent(b->cl_st[k], b->cl_ev[5], 0));
    CK(c, launch_gdp_cluster(q.C, q.threads, P.irp, b->d_pk, b->d_cl_list + off[k], cnt, P.ilam[0],
                             c->p.damping_shift, c->p.max_iters, b->d_cl_out, q.emax, q.nmax,
                             b->cl_st[k]));
    CK(c, cudaEventRecord(b->cl_ev[k], b->cl_st[k]));
    CK(c, cudaStreamWaitEvent(c->st, b->cl_ev[k], 0));
  }
  CK(c, cudaEventRecord(c->ev1, c->st));
  CK(c, cudaMemcpyAsync(b->h_cl_out, b->d_cl_out, sizeof(ClusterOut) * K, cudaMemcpyDeviceToHost, c->st));
  CK(c, scatter_perm(P.ilam[0], P.perm, c->n, c->d_lam[c->cur], c->st));
  CK(c, cudaStreamSynchronize(c->st));
  float t_ms = 0.f;
  cudaEventElapsedTime(&t_ms, c->ev0, c->ev1);
  if (ms) *ms += t_ms;
  int st = 0;
  for (int32_t s = 0; s < K; ++s) {
    if (!active[s]) continue;
    st |= b->h_cl_out[s].status;
    sweeps_out[s] += b->h_cl_out[s].sweeps;
  }
  if (st & kGdpOverflow) return fail(c, F2M_ERR_OVERFLOW, "|lambda| reached 2^29 in some instance");
  return F2M_OK;
}

static f2m_status batch_gdp_phase(f2m_batch* b, const std::vector<uint8_t>& active,
                                  std::vector<int64_t>& sweeps_out, double* ms) {
  f2m_ctx* c = b->u;
  c->lam_version += 1;
  GdpPlan& P = c->plan;
  const int32_t F = c->p.frac_bits;
  if (c->fb_cur != F) {  // continue from the finisher's lambda: floor to F bits
    CK(c, launch_halve(c->d_lam2, c->d_lam[c->cur], c->n, c->st));
    c->fb_cur = F;
  }
  // clusters when asked for, unless a streaming-kernel shape is given or some
  // instance does not fit a cluster
  b->used_clusters = false;
  if (c->p.batch_shape < 0 && (c->p.flags & F2M_FLAG_BATCH_CLUSTERS)) {
    if (b->cl_version != P.version) {
      f2m_status s = cluster_plan(b);
      if (s != F2M_OK) return s;
    }
    if (b->cl_ok) {
      b->used_clusters = true;
      return batch_cluster_phase(b, active, sweeps_out, ms);
    }
  }
  if (b->tiles_version != P.version) {
    f2m_status s = F2M_OK;
    if (c->p.batch_shape >= 0) {
      b->shape = c->p.batch_shape;
    } else if (b->shape < 0) {
      s = batch_autotune(b);
      if (s != F2M_OK) return s;
    }
    int te = 0, tn = 0;
    batch_shape_tile(b->shape, &te, &tn);
    s = batch_tiles(b, te, tn, b->tiles_all, b->e1_all);
    if (s != F2M_OK) return s;
    s = batch_list_reserve(b, (int32_t)b->tiles_all.size());
    if (s != F2M_OK) return s;
    b->grid = batch_grid(b, b->shape, (int32_t)b->tiles_all.size());
    if (b->grid < 1) return fail(c, F2M_ERR_CUDA, "the batch kernel shape does not fit an SM");
    b->tiles_version = P.version;
  }
  const int32_t max_tiles = (int32_t)b->tiles_all.size();
  std::memcpy(b->h_active, active.data(), b->count);
  CK(c, enqueue_phase_start(b, c->st, b->h_active));
  // capture one launch once per tile version; every launch of every phase replays it
  const bool graph = c->p.batch_graph && !b->graph_failed;
  if (graph && (!b->gexec || b->graph_version != b->tiles_version)) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    CK(c, cudaStreamSynchronize(c->st));
    const long long before = f2m_kernel_launches();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e2 = enqueue_launch(b, b->gs, b->shape, b->grid, max_tiles);
      e = cudaStreamEndCapture(b->gs, &g);
      if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    b->graph_kernels = f2m_kernel_launches() - before;
    count_launches(-b->graph_kernels);  // captured, not launched
    if (e != cudaSuccess) {  // capture not available here: launch directly from now on
      cudaGetLastError();
      if (b->gexec) cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
      b->graph_failed = true;
    } else {
      b->graph_version = b->tiles_version;
    }
  }
  std::vector<uint8_t> act(active.begin(), active.end());
  long long t_base = 0;
  for (;;) {
    const int32_t nt = fill_list(b, b->tiles_all, b->e1_all, act.data());
    const long long left = c->p.max_iters - t_base;
    *b->h_chunk = BatchChunk{nt, 0, t_base, left < kSweepsPerLaunch ? left : kSweepsPerLaunch};
    if (b->gexec) {
      CK(c, cudaEventRecord(b->e_in, c->st));
      CK(c, cudaStreamWaitEvent(b->gs, b->e_in, 0));
      CK(c, cudaEventRecord(c->ev0, b->gs));
      CK(c, cudaGraphLaunch(b->gexec, b->gs));
      CK(c, cudaEventRecord(c->ev1, b->gs));
      CK(c, cudaEventRecord(b->e_out, b->gs));
      CK(c, cudaStreamWaitEvent(c->st, b->e_out, 0));
      count_launches(b->graph_kernels);
    } else {
      CK(c, cudaEventRecord(c->ev0, c->st));
      CK(c, enqueue_launch(b, c->st, b->shape, b->grid, max_tiles));
      CK(c, cudaEventRecord(c->ev1, c->st));
    }
    CK(c, cudaStreamSynchronize(c->st));
    float t_ms = 0.f;
    cudaEventElapsedTime(&t_ms, c->ev0, c->ev1);
    if (ms) *ms += t_ms;
    const GdpCtl h = *b->h_ctl;
    if (h.status & kGdpTimeout) return fail(c, F2M_ERR_TIMEOUT, "device-wide barrier wait exceeded its budget");
    if (h.status & kGdpOverflow) return fail(c, F2M_ERR_OVERFLOW, "|lambda| reached 2^29 in some instance");
    bool any = false;
    for (int32_t s = 0; s < b->count; ++s) {
      if (!act[s]) continue;
      if (!b->h_still[s]) {
        sweeps_out[s] += b->h_sw[s];  // froze in this launch (the record includes t_base)
        act[s] = 0;
      } else {
        any = true;
      }
    }
    t_base += h.sweeps;
    const bool more = any && !h.fixed_point && t_base < c->p.max_iters && (h.sweeps & 1) == 0;
    if (!more) {
      for (int32_t s = 0; s < b->count; ++s)
        if (act[s]) sweeps_out[s] += t_base;  // ran to the cap
      break;
    }
  }
  // lambda back to caller order from the buffer the last launch ended in
  CK(c, launch_batch_scatter_final(P.ilam[0], P.ilam[1], c->d_gdp, P.perm, c->n, c->d_lam[c->cur], c->st));
  return F2M_OK;
}

// Copy the results of the instances flagged in `done` out of the union state.
static f2m_status snapshot(f2m_batch* b, const std::vector<uint8_t>& done) {
  f2m_ctx* c = b->u;
  const int32_t K = b->count;
  int32_t fb = 0;
  const int32_t* lam = cur_lambda(c, &fb);
  if (!b->h_snap) {  // pinned staging: bounds and entry offsets down, mask and arena offsets up
    CK(c, cudaMallocHost((void**)&b->h_snap, sizeof(long long) * K + sizeof(int32_t) * (K + 1) +
                                              sizeof(long long) * K + K));
    CK(c, dalloc(&b->d_snap_eoff, K));
    CK(c, dalloc(&b->d_snap_done, K));
    CK(c, dalloc(&b->d_snap_ent, K + 1));
  }
  long long* h_b2 = b->h_snap;
  int32_t* h_ent = reinterpret_cast<int32_t*>(h_b2 + K);
  long long* h_eoff = reinterpret_cast<long long*>(h_ent + K + 1);
  uint8_t* h_done = reinterpret_cast<uint8_t*>(h_eoff + K);
  CK(c, launch_batch_extract_bound(c->d_rp, c->d_ec, lam, c->n, fb, c->d_seg_off, K, c->d_x2,
                                   b->d_seg_b2, b->d_seg_bad, nullptr, c->st));
  CK(c, launch_batch_seg_entry(c->d_rp, c->d_seg_off, K, b->d_snap_ent, c->st));
  CK(c, cudaMemcpyAsync(h_b2, b->d_seg_b2, sizeof(long long) * K, cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaMemcpyAsync(h_ent, b->d_snap_ent, sizeof(int32_t) * (K + 1), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  int64_t need = b->res_used;
  for (int32_t s = 0; s < K; ++s)
    if (done[s]) need += h_ent[s + 1] - h_ent[s];
  if (need > b->res_cap) {  // grow the arenas, keeping what they hold
    const int64_t cap = need + (need >> 2) + 1024;
    int2* ec = nullptr;
    uint8_t* x2 = nullptr;
    CK(c, dalloc(&ec, cap));
    CK(c, dalloc(&x2, cap));
    if (b->res_used) {
      CK(c, cudaMemcpyAsync(ec, b->d_res_ec, sizeof(int2) * b->res_used, cudaMemcpyDeviceToDevice, c->st));
      CK(c, cudaMemcpyAsync(x2, b->d_res_x2, b->res_used, cudaMemcpyDeviceToDevice, c->st));
      CK(c, cudaStreamSynchronize(c->st));
    }
    dfree(b->d_res_ec);
    dfree(b->d_res_x2);
    b->d_res_ec = ec;
    b->d_res_x2 = x2;
    b->res_cap = cap;
  }
  bool any = false;
  for (int32_t s = 0; s < K; ++s) {
    h_done[s] = done[s];
    h_eoff[s] = 0;
    if (!done[s]) continue;
    any = true;
    const int64_t nz = h_ent[s + 1] - h_ent[s];
    h_eoff[s] = b->res_used;
    b->res_eoff[s] = b->res_used;
    b->res_nnz[s] = nz;
    b->res_b2[s] = h_b2[s];
    b->res_fb[s] = fb;
    b->res_done[s] = 1;
    b->res_used += nz;
  }
  if (!any) return F2M_OK;
  CK(c, cudaMemcpyAsync(b->d_snap_done, h_done, K, cudaMemcpyHostToDevice, c->st));
  CK(c, cudaMemcpyAsync(b->d_snap_eoff, h_eoff, sizeof(long long) * K, cudaMemcpyHostToDevice, c->st));
  CK(c, launch_batch_snapshot(b->d_snap_done, c->d_seg_off, K, c->d_rp, lam, c->d_ec, c->d_x2, b->d_snap_eoff,
                              b->d_res_lam, b->d_res_rp, b->d_res_ec, b->d_res_x2, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return F2M_OK;
}

// The solve loop of f2m_solve, kept per instance; every device step covers
// all instances that are at that step.
extern "C" f2m_status f2m_solve_batch(f2m_batch* b, f2m_info* info_out, f2m_info* total_out) {
  if (!b) return fail(nullptr, F2M_ERR_INVALID_ARG, "NULL batch");
  f2m_ctx* c = b->u;
  const auto t0 = std::chrono::steady_clock::now();
  const int32_t K = b->count;
  enum { GDP = 0, EXTRACT = 1, DONE = 2 };
  std::vector<int> state(K, GDP);
  std::vector<uint8_t> clean(K, 0), active(K, 0), include(K, 0), done_now(K, 0);
  std::vector<int64_t> sweeps(K, 0), phases(K, 0), rounds(K, 0), added(K, 0), fin_calls(K, 0);
  std::vector<int64_t> last_pairs(K, 0);  // pairs found by each instance's last scan
  std::vector<int32_t> certified(K, 0), inst_status(K, F2M_OK);
  b->res_eoff.assign(K, 0);
  b->res_nnz.assign(K, 0);
  b->res_b2.assign(K, 0);
  b->res_fb.assign(K, c->p.frac_bits);
  b->res_done.assign(K, 0);
  b->res_used = 0;
  f2m_info tot;
  std::memset(&tot, 0, sizeof(tot));
  c->fin_stats = FinisherStats();
  f2m_status status = F2M_OK;
  auto any_in = [&](int st) {
    for (int s : state)
      if (s == st) return true;
    return false;
  };
  while (status == F2M_OK && (any_in(GDP) || any_in(EXTRACT))) {
    if (any_in(GDP)) {
      for (int32_t s = 0; s < K; ++s) active[s] = state[s] == GDP;
      status = batch_gdp_phase(b, active, sweeps, &tot.ms_gdp);
      if (status != F2M_OK) break;
      tot.phases += 1;
      c->seg_scan.assign(K, 0);
      bool any_scan = false;
      for (int32_t s = 0; s < K; ++s) {
        if (!active[s]) continue;
        phases[s] += 1;
        clean[s] = 0;
        // as f2m_solve: price after the first phase and after a phase whose
        // preceding scan found at least n/1024 pairs
        if (c->p.pricing && rounds[s] < c->p.max_pricing_rounds &&
            (phases[s] == 1 || last_pairs[s] * 1024 >= b->n[s])) {
          c->seg_scan[s] = 1;
          any_scan = true;
        } else {
          state[s] = EXTRACT;
        }
      }
      if (any_scan) {  // pricing with the GDP lambda
        status = price_internal(c, &tot.ms_pricing);
        tot.pricing_pairs += c->last_scan_pairs;
        if (status != F2M_OK) break;
        tot.pricing_rounds += 1;
        for (int32_t s = 0; s < K; ++s) {
          if (!c->seg_scan[s]) continue;
          rounds[s] += 1;
          last_pairs[s] = c->seg_pairs[s];
          if (c->seg_pairs[s] > 0) {
            added[s] += c->seg_pairs[s];
            // another GDP phase, unless the first phase's scan found few
            // pairs (as f2m_solve): the finisher takes them from this lambda
            if (phases[s] == 1 && c->seg_pairs[s] * 1024 < b->n[s]) state[s] = EXTRACT;
          } else {
            clean[s] = 1;
            state[s] = EXTRACT;
          }
        }
        if (c->npairs > 0) {
          status = merge_internal(c, c->d_pairs, c->npairs, &tot.ms_merge);
          if (status != F2M_OK) break;
          tot.edges_added += c->npairs;
        }
      }
      if (any_in(GDP)) continue;  // the others wait at EXTRACT
    }
    // rule (7) for the instances at EXTRACT; the finisher for those with defects
    int32_t fb = 0;
    const int32_t* lam = cur_lambda(c, &fb);
    for (int32_t s = 0; s < K; ++s) done_now[s] = state[s] == EXTRACT;
    CK(c, cudaMemcpyAsync(b->d_mask, done_now.data(), K, cudaMemcpyHostToDevice, c->st));
    CK(c, cudaEventRecord(c->ev0, c->st));
    CK(c, launch_batch_extract_bound(c->d_rp, c->d_ec, lam, c->n, fb, c->d_seg_off, K, c->d_x2,
                                     b->d_seg_b2, b->d_seg_bad, b->d_mask, c->st));
    CK(c, cudaEventRecord(c->ev1, c->st));
    std::vector<unsigned long long> bad(K);
    CK(c, cudaMemcpyAsync(bad.data(), b->d_seg_bad, sizeof(unsigned long long) * K, cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev0, c->ev1);
      tot.ms_extract += ms;
    }
    bool any_bad = false;
    for (int32_t s = 0; s < K; ++s) {
      include[s] = state[s] == EXTRACT && bad[s] > 0;
      any_bad |= include[s] != 0;
    }
    if (any_bad) {
      if (!c->p.finisher) {
        status = F2M_ERR_NOT_CONVERGED;
        fail(c, status, "some instance violates the degree constraint and the finisher is off");
        break;
      }
      CK(c, cudaMemcpyAsync(c->d_fin_include, include.data(), K, cudaMemcpyHostToDevice, c->st));
      const auto f0 = std::chrono::steady_clock::now();
      int64_t aug = 0;
      status = finisher_internal(c, &aug, include.data());
      tot.ms_finish += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - f0).count();
      if (status != F2M_OK) break;
      tot.finisher_calls += 1;
      tot.augmentations += aug;
      for (int32_t s = 0; s < K; ++s) fin_calls[s] += include[s];
    }
    // pricing with the final lambda where it changed since the clean scan
    c->seg_scan.assign(K, 0);
    bool any_scan = false;
    std::fill(done_now.begin(), done_now.end(), 0);
    for (int32_t s = 0; s < K; ++s) {
      if (state[s] != EXTRACT) continue;
      certified[s] = 1;
      if (!c->p.pricing) { done_now[s] = 1; continue; }
      if (clean[s] && !include[s]) { certified[s] = 2; done_now[s] = 1; continue; }
      if (rounds[s] >= c->p.max_pricing_rounds) {
        done_now[s] = 1;
        inst_status[s] = F2M_ERR_NOT_CONVERGED;
        continue;
      }
      c->seg_scan[s] = 1;
      any_scan = true;
    }
    if (any_scan) {
      status = price_internal(c, &tot.ms_pricing);
      tot.pricing_pairs += c->last_scan_pairs;
      if (status != F2M_OK) break;
      tot.pricing_rounds += 1;
      for (int32_t s = 0; s < K; ++s) {
        if (!c->seg_scan[s]) continue;
        rounds[s] += 1;
        last_pairs[s] = c->seg_pairs[s];
        if (c->seg_pairs[s] == 0) {
          certified[s] = 2;
          done_now[s] = 1;
        } else {
          added[s] += c->seg_pairs[s];
          certified[s] = 0;
          state[s] = GDP;
        }
      }
    }
    status = snapshot(b, done_now);  // before merges move the entries
    if (status != F2M_OK) break;
    for (int32_t s = 0; s < K; ++s)
      if (done_now[s]) state[s] = DONE;
    if (any_scan && c->npairs > 0) {
      status = merge_internal(c, c->d_pairs, c->npairs, &tot.ms_merge);
      if (status != F2M_OK) break;
      tot.edges_added += c->npairs;
    }
  }
  CK(c, cudaMemsetAsync(c->d_fin_include, 1, K, c->st));
  c->seg_scan.clear();
  CK(c, cudaStreamSynchronize(c->st));
  for (int32_t s = 0; s < K; ++s) {
    tot.iterations += sweeps[s];
    tot.bound2 += b->res_b2[s];
  }
  tot.frac_bits = -1;  // per instance
  tot.nnz = b->res_used;
  tot.batch_shape = b->shape;
  tot.batch_graph = b->gexec != nullptr ? 1 : 0;
  tot.gdp_kernel = b->used_clusters ? F2M_GDP_KERNEL_BATCH_CLUSTERS : F2M_GDP_KERNEL_BATCH;
  tot.certified = 2;
  for (int32_t s = 0; s < K; ++s) {
    tot.certified = std::min(tot.certified, certified[s]);
    if (status == F2M_OK && inst_status[s] != F2M_OK) status = (f2m_status)inst_status[s];
  }
  tot.status = status;
  copy_finisher_stats(c, &tot);
  tot.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info_out) {
    for (int32_t s = 0; s < K; ++s) {
      f2m_info& f = info_out[s];
      std::memset(&f, 0, sizeof(f));
      f.iterations = sweeps[s];
      f.phases = phases[s];
      f.pricing_rounds = rounds[s];
      f.edges_added = added[s];
      f.finisher_calls = fin_calls[s];
      f.augmentations = -1;  // counted for the whole batch only
      f.bound2 = b->res_b2[s];
      f.frac_bits = b->res_fb[s];
      f.certified = certified[s];
      f.status = status == F2M_OK ? inst_status[s] : status;
      f.nnz = b->res_nnz[s];
      f.batch_shape = -1;
    }
  }
  if (total_out) *total_out = tot;
  return status;
}

static f2m_status stage(f2m_batch* b, int64_t cap) {
  f2m_ctx* c = b->u;
  if (b->tmp_cap >= cap) return F2M_OK;
  dfree(b->d_tmp_a);
  dfree(b->d_tmp_b);
  CK(c, dalloc(&b->d_tmp_a, cap));
  CK(c, dalloc(&b->d_tmp_b, cap));
  b->tmp_cap = cap;
  return F2M_OK;
}

__global__ void f2m_offset_kernel(const int32_t* __restrict__ in, int64_t count, int32_t sub,
                                  int32_t* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i] - sub;
}

extern "C" f2m_status f2m_batch_get_lambda(f2m_batch* b, int32_t i, int32_t* lambda, int32_t* frac_bits) {
  if (!b || i < 0 || i >= b->count) return bfail(b, F2M_ERR_INVALID_ARG, "bad batch or index");
  if ((int32_t)b->res_done.size() != b->count || !b->res_done[i])
    return bfail(b, F2M_ERR_INVALID_ARG, "instance has no result yet");
  f2m_ctx* c = b->u;
  if (frac_bits) *frac_bits = b->res_fb[i];
  if (lambda) {
    CK(c, cudaMemcpyAsync(lambda, b->d_res_lam + c->seg_off[i], sizeof(int32_t) * b->n[i], cudaMemcpyDefault, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return F2M_OK;
}

extern "C" f2m_status f2m_batch_get_x(f2m_batch* b, int32_t i, int64_t* nnz_inout, int32_t* row_ptr,
                                      int32_t* col, uint8_t* x2) {
  if (!b || i < 0 || i >= b->count || !nnz_inout) return bfail(b, F2M_ERR_INVALID_ARG, "bad batch or index");
  if ((int32_t)b->res_done.size() != b->count || !b->res_done[i])
    return bfail(b, F2M_ERR_INVALID_ARG, "instance has no result yet");
  f2m_ctx* c = b->u;
  const int64_t nz = b->res_nnz[i];
  const int64_t cap = *nnz_inout;
  *nnz_inout = nz;
  if (!row_ptr && !col && !x2) return F2M_OK;
  if ((col || x2) && cap < nz) return bfail(b, F2M_ERR_INVALID_ARG, "capacity below nnz");
  f2m_status s = stage(b, std::max<int64_t>(nz, b->n[i] + 1));
  if (s != F2M_OK) return s;
  const int32_t* rp = b->d_res_rp + c->seg_off[i] + i;
  if (row_ptr) {
    int32_t r0 = 0;
    CK(c, cudaMemcpyAsync(&r0, rp, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    f2m_offset_kernel<<<64, 256, 0, c->st>>>(rp, b->n[i] + 1, r0, b->d_tmp_a);
    count_launch();
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(row_ptr, b->d_tmp_a, sizeof(int32_t) * (b->n[i] + 1), cudaMemcpyDefault, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  if (col && nz) {
    CK(c, launch_split_ec(b->d_res_ec + b->res_eoff[i], nz, b->d_tmp_b, nullptr, c->st));
    f2m_offset_kernel<<<256, 256, 0, c->st>>>(b->d_tmp_b, nz, c->seg_off[i], b->d_tmp_a);
    count_launch();
    CK(c, cudaGetLastError());
    CK(c, cudaMemcpyAsync(col, b->d_tmp_a, sizeof(int32_t) * nz, cudaMemcpyDefault, c->st));
  }
  if (x2 && nz) CK(c, cudaMemcpyAsync(x2, b->d_res_x2 + b->res_eoff[i], nz, cudaMemcpyDefault, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return F2M_OK;
}

extern "C" const char* f2m_batch_last_error(const f2m_batch* b) {
  return f2m_last_error(b ? b->u : nullptr);
}
