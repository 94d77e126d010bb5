// C ABI of the f2m library (declared in include/f2m.h): context, input
// validation, the hot-path step calls and the solve driver.
//
// The driver runs on the host and only sequences device work: every GDP sweep,
// pricing test, merge and extraction runs in this library's kernels on the
// context's stream; the host reads back one small status block per step.  The
// exception is the exact finisher (finisher.cpp), a min-cost flow that runs on
// the host when the sign rule (7) leaves some node with a row sum other than 2.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <climits>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/f2m.h"
#include "ctx_internal.h"
#include "f2m_internal.h"

using namespace f2m;

static std::atomic<long long> g_kernel_launches{0};

namespace f2m {
void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long k) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace f2m

extern "C" int64_t f2m_kernel_launches(void) { return g_kernel_launches.load(); }



// Pinned host blocks are costly to allocate (about a millisecond for the
// finisher's mirrors of a 100k-node graph), so freed blocks are kept for the
// next context, up to 2 GiB; a block is reused for a request of at least half
// its size.
namespace {
std::mutex g_pin_mu;
std::multimap<size_t, void*> g_pin_free;       // size -> cached block
std::map<void*, size_t> g_pin_size;            // every block handed out or cached
size_t g_pin_cached = 0;
constexpr size_t kPinCacheMax = (size_t)1 << 31;

cudaError_t pin_alloc(void** p, size_t bytes) {
  if (bytes == 0) bytes = 1;
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    auto it = g_pin_free.lower_bound(bytes);
    if (it != g_pin_free.end() && it->first <= 2 * bytes) {
      *p = it->second;
      g_pin_cached -= it->first;
      g_pin_free.erase(it);
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaMallocHost(p, bytes);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_size[*p] = bytes;
  }
  return e;
}

void pin_free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  auto it = g_pin_size.find(p);
  if (it == g_pin_size.end()) return;
  if (g_pin_cached + it->second <= kPinCacheMax) {
    g_pin_free.emplace(it->second, p);
    g_pin_cached += it->second;
  } else {
    cudaFreeHost(p);
    g_pin_size.erase(it);
  }
}

// Device blocks: creating a context makes about sixty allocations, each
// costing more than the kernel that fills it, so freed blocks are kept per
// device (up to 4 GiB each) and reused for a request of at least half their
// size.  A block enters the cache only after the device has finished all
// work queued before its release (as cudaFree would wait), so no kernel still
// in flight can see it handed out again.
struct DevBlock {
  size_t bytes;
  int device;
};
std::mutex g_dev_mu;
std::multimap<std::pair<int, size_t>, void*> g_dev_free;  // (device, size) -> cached block
std::map<void*, DevBlock> g_dev_size;                      // every block handed out or cached
std::map<int, size_t> g_dev_cached;
constexpr size_t kDevCacheMax = (size_t)1 << 32;

void dev_cache_flush(int dev) {  // caller holds g_dev_mu
  for (auto it = g_dev_free.begin(); it != g_dev_free.end();) {
    if (it->first.first == dev) {
      cudaFree(it->second);
      g_dev_size.erase(it->second);
      it = g_dev_free.erase(it);
    } else {
      ++it;
    }
  }
  g_dev_cached[dev] = 0;
}

void dev_release_locked(void* p) {
  auto it = g_dev_size.find(p);
  if (it == g_dev_size.end()) {  // not ours: a plain block
    cudaFree(p);
    return;
  }
  const DevBlock b = it->second;
  size_t& cached = g_dev_cached[b.device];
  if (cached + b.bytes <= kDevCacheMax) {
    g_dev_free.emplace(std::make_pair(b.device, b.bytes), p);
    cached += b.bytes;
  } else {
    cudaFree(p);
    g_dev_size.erase(it);
  }
}
}  // namespace

namespace f2m {

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (bytes == 0) bytes = 1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_dev_free.lower_bound(std::make_pair(dev, bytes));
  if (it != g_dev_free.end() && it->first.first == dev && it->first.second <= 2 * bytes) {
    *p = it->second;
    g_dev_cached[dev] -= it->first.second;
    g_dev_free.erase(it);
    return cudaSuccess;
  }
  e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {  // give the cached blocks back and try again
    cudaGetLastError();
    dev_cache_flush(dev);
    e = cudaMalloc(p, bytes);
  }
  if (e == cudaSuccess) g_dev_size[*p] = DevBlock{bytes, dev};
  return e;
}

static thread_local int t_dev_synced = 0;  // > 0 inside a DevSyncedScope

DevSyncedScope::DevSyncedScope() {
  cudaDeviceSynchronize();
  ++t_dev_synced;
}
DevSyncedScope::~DevSyncedScope() { --t_dev_synced; }

void dev_free(void* p) {
  if (!p) return;
  if (!t_dev_synced) cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  dev_release_locked(p);
}

void dev_free_synced(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  dev_release_locked(p);
}

}  // namespace f2m

// The host's pinned copies of the finisher's input and output (row offsets,
// entries, twins, flow, surpluses, lambda): one set for the process, taken by
// one finisher call at a time.  Contexts that each kept their own set touched
// tens of MB of pinned pages apiece, and the device's copies into pages it had
// not touched lately ran several times slower than into recently used ones;
// one set stays in use.  `owner` is the context whose graph the entry arrays
// hold (its fin_version says at which version); any other context copies its
// graph again.
struct HostMirror {
  std::mutex mu;
  int32_t* irp = nullptr;
  int2* iec = nullptr;
  int32_t* twin = nullptr;
  uint8_t* y = nullptr;
  int32_t* exl = nullptr;
  int32_t* lam = nullptr;
  int32_t* lam2 = nullptr;
  int64_t cap = 0;    // entries
  int64_t ncap = 0;   // nodes
  const f2m_ctx* owner = nullptr;
};
static HostMirror g_mirror;

// takes the mirror for context c (lock held by the caller) with room for its
// graph; points c's host arrays at it
static cudaError_t take_mirror(f2m_ctx* c) {
  HostMirror& M = g_mirror;
  const int64_t cap = std::max<int64_t>(c->fin_cap, c->nnz);
  if (M.cap < cap || M.ncap < (int64_t)c->n + 1) {
    const int64_t ec = std::max<int64_t>(cap, M.cap), nc = std::max<int64_t>((int64_t)c->n + 1, M.ncap);
    void* old[] = {M.irp, M.iec, M.twin, M.y, M.exl, M.lam, M.lam2};
    for (void* q : old) pin_free(q);
    M.irp = nullptr; M.iec = nullptr; M.twin = nullptr; M.y = nullptr;
    M.exl = nullptr; M.lam = nullptr; M.lam2 = nullptr;
    M.cap = M.ncap = 0;
    M.owner = nullptr;
    cudaError_t e = pin_alloc((void**)&M.iec, sizeof(int2) * ec);
    if (e == cudaSuccess) e = pin_alloc((void**)&M.twin, sizeof(int32_t) * ec);
    if (e == cudaSuccess) e = pin_alloc((void**)&M.y, ec);
    if (e == cudaSuccess) e = pin_alloc((void**)&M.irp, sizeof(int32_t) * nc);
    if (e == cudaSuccess) e = pin_alloc((void**)&M.exl, sizeof(int32_t) * nc);
    if (e == cudaSuccess) e = pin_alloc((void**)&M.lam, sizeof(int32_t) * nc);
    if (e == cudaSuccess) e = pin_alloc((void**)&M.lam2, sizeof(int32_t) * nc);
    if (e != cudaSuccess) return e;
    M.cap = ec;
    M.ncap = nc;
  }
  if (M.owner != c) {
    c->fin_version = -1;  // the entry arrays hold another graph
    M.owner = c;
  }
  c->h_irp = M.irp; c->h_iec = M.iec; c->h_twin = M.twin; c->h_y = M.y;
  c->h_exl = M.exl; c->h_lam = M.lam; c->h_lam2 = M.lam2;
  return cudaSuccess;
}

static void free_finisher_buffers(f2m_ctx* c) {
  dev_free(c->d_twin);
  dev_free(c->d_fy);
  dfree(c->d_fpi); dfree(c->d_fdist); dfree(c->d_fex); dfree(c->d_fvia); dfree(c->d_fpred);
  dfree(c->d_freach); dfree(c->d_fclos); dfree(c->d_forder); dfree(c->d_fstat); dfree(c->d_fblk);
  dfree(c->d_fcaps); dfree(c->d_fheap_off); dfree(c->d_fpush); dfree(c->d_fheap);
  pin_free(c->h_fpi);
  pin_free(c->h_fex);
  c->h_fpi = nullptr;
  c->h_fex = nullptr;
  c->fblk_cap = 0;
  c->fheap_cap = 0;
  {
    std::lock_guard<std::mutex> lk(g_mirror.mu);
    if (g_mirror.owner == c) g_mirror.owner = nullptr;  // a later context may sit at this address
  }
  c->d_twin = nullptr; c->d_fy = nullptr;
  c->h_irp = nullptr; c->h_iec = nullptr; c->h_twin = nullptr; c->h_y = nullptr;
  c->h_exl = nullptr; c->h_lam = nullptr; c->h_lam2 = nullptr;
  c->fin_cap = 0;
  c->fin_version = -1;
  c->twin_version = -1;
}

// device buffers for `cap` entries (the host side is the process's mirror,
// taken per finisher call)
static cudaError_t alloc_finisher_buffers(f2m_ctx* c, int64_t cap) {
  dev_free(c->d_twin);
  dev_free(c->d_fy);
  c->d_twin = nullptr; c->d_fy = nullptr;
  c->fin_cap = 0;
  c->fin_version = -1;
  c->twin_version = -1;
  cudaError_t e = dev_malloc((void**)&c->d_twin, sizeof(int32_t) * cap);
  if (e == cudaSuccess) e = dev_malloc((void**)&c->d_fy, cap);
  if (e == cudaSuccess) c->fin_cap = cap;
  return e;
}

static thread_local std::string g_create_error;

namespace f2m {

f2m_status fail(f2m_ctx* ctx, f2m_status s, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_create_error = msg;
  return s;
}

f2m_status cuda_fail(f2m_ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(ctx, F2M_ERR_OOM, m);
  return fail(ctx, F2M_ERR_CUDA, m);
}

}  // namespace f2m

static float elapsed_ms(f2m_ctx* c) {
  float ms = 0.f;
  cudaEventSynchronize(c->ev1);
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  return ms;
}

extern "C" void f2m_default_params(f2m_params* p) {
  if (!p) return;
  p->frac_bits = 8;
  p->damping_shift = 2;
  p->max_iters = 128;
  p->max_pricing_rounds = 64;
  p->pricing = 1;
  p->pricing_cap = 1 << 20;
  p->barrier_budget_cycles = 4000000000LL;
  p->finisher = 1;
  p->flags = 0;
  p->gdp_lanes = 0;
  p->gdp_ctas_per_sm = 0;
  p->batch_shape = -1;
  p->batch_graph = 1;
}

extern "C" const char* f2m_status_string(f2m_status s) {
  switch (s) {
    case F2M_OK: return "ok";
    case F2M_ERR_INVALID_ARG: return "invalid argument";
    case F2M_ERR_CUDA: return "CUDA error";
    case F2M_ERR_OOM: return "out of memory";
    case F2M_ERR_NOT_CONVERGED: return "not converged";
    case F2M_ERR_OVERFLOW: return "lambda overflow";
    case F2M_ERR_PRICING_OVERFLOW: return "pricing buffer overflow";
    case F2M_ERR_INFEASIBLE: return "infeasible";
    case F2M_ERR_TIMEOUT: return "device barrier timeout";
  }
  return "unknown status";
}

extern "C" const char* f2m_last_error(const f2m_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" void f2m_destroy(f2m_ctx* c) {
  if (!c) return;
  DevSyncedScope synced;  // one wait for the device, then every block goes to the cache
  dfree(c->d_xy); dfree(c->d_rp); dfree(c->d_ec); dfree(c->d_ec_alt); dfree(c->d_x2); dfree(c->d_tiles);
  dfree(c->d_seg_off); dfree(c->d_fin_include);
  dfree(c->d_lam[0]); dfree(c->d_lam[1]); dfree(c->d_lam2); dfree(c->d_exl); dfree(c->d_gdp);
  dfree(c->d_trace_b2); dfree(c->d_trace_ch); dfree(c->d_pts); dfree(c->d_pairs);
  dfree(c->d_pts4); dfree(c->d_pstat); dfree(c->d_mranges); dfree(c->d_mtblk); dfree(c->d_mbox);
  dfree(c->d_mlmax); dfree(c->d_mframes); dfree(c->d_mcand); dfree(c->d_mncand);
  dfree(c->d_lam_ref); dfree(c->d_raised); dfree(c->d_pts_raised); dfree(c->d_nraised);
  dfree(c->d_ranges); dfree(c->d_boxes); dfree(c->d_smax);
  dfree(c->d_count); dfree(c->d_tile); dfree(c->d_deg); dfree(c->d_tmp_rp); dfree(c->d_new_rp);
  dfree(c->d_block_sums); dfree(c->d_tmp_col); dfree(c->d_out_a); dfree(c->d_out_b);
  dfree(c->d_check); dfree(c->d_scalar); dfree(c->d_bad); dfree(c->d_b); dfree(c->d_b_int);
  free_finisher_buffers(c);
  if (c->fin_work) finisher_work_free(c->fin_work);
  plan2_free(c->plan);
  plan_free(c->plan);
  class_plan_free(c->classes);
  cut_state_free(c->cuts);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

f2m_status f2m::check_params_internal(const f2m_params& p) {
  if (p.frac_bits < 1 || p.frac_bits > 8) return fail(nullptr, F2M_ERR_INVALID_ARG, "frac_bits must be in 1..8");
  if (p.damping_shift < 1 || p.damping_shift > 8) return fail(nullptr, F2M_ERR_INVALID_ARG, "damping_shift must be in 1..8");
  if (p.gdp_lanes != 0 && p.gdp_lanes != 1)
    return fail(nullptr, F2M_ERR_INVALID_ARG, "gdp_lanes must be 0 or 1");
  if (p.gdp_ctas_per_sm < 0 || p.gdp_ctas_per_sm > 2)
    return fail(nullptr, F2M_ERR_INVALID_ARG, "gdp_ctas_per_sm must be 0, 1 or 2");
  if (p.batch_shape < -1 || p.batch_shape >= batch_num_shapes())
    return fail(nullptr, F2M_ERR_INVALID_ARG, "batch_shape must be -1 or a shape index");
  if (p.batch_graph != 0 && p.batch_graph != 1)
    return fail(nullptr, F2M_ERR_INVALID_ARG, "batch_graph must be 0 or 1");
  if (p.max_iters < 0 || p.max_pricing_rounds < 0 || p.pricing_cap < 1 || p.barrier_budget_cycles < 0)
    return fail(nullptr, F2M_ERR_INVALID_ARG, "negative cap or budget");
  if (p.pricing < 0 || p.pricing > 2) return fail(nullptr, F2M_ERR_INVALID_ARG, "pricing must be 0, 1 or 2");
  return F2M_OK;
}

static std::string check_message(int flags, int first) {
  static const char* names[] = {"row_ptr not monotone or not ending at nnz", "column index out of range",
                                "row not sorted ascending or duplicate column", "self-loop",
                                "CSR not symmetric", "node degree below 3",
                                "coordinate outside [0, 2^20)", "pair out of range or u == v",
                                "degree requirement b_v outside [1, deg(v) - 1]"};
  std::string m;
  for (int b = 0; b < 9; ++b)
    if (flags & (1 << b)) {
      if (!m.empty()) m += "; ";
      m += names[b];
    }
  return m + " (first at index " + std::to_string(first) + ")";
}

static cudaError_t reset_check(f2m_ctx* c) {
  CheckCtl h{0, INT_MAX};
  return cudaMemcpyAsync(c->d_check, &h, sizeof(h), cudaMemcpyHostToDevice, c->st);
}

static cudaError_t read_check(f2m_ctx* c, CheckCtl* h) {
  cudaError_t e = cudaMemcpyAsync(h, c->d_check, sizeof(*h), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return e;
}

extern "C" f2m_status f2m_create(const int32_t* xy, int32_t n, const int32_t* row_ptr,
                                 const int32_t* col, const f2m_params* params, void* stream,
                                 f2m_ctx** out) {
  return create_internal(xy, n, row_ptr, col, params, stream, std::vector<int32_t>{0, n}, out);
}

f2m_status f2m::create_internal(const int32_t* xy, int32_t n, const int32_t* row_ptr,
                                const int32_t* col, const f2m_params* params, void* stream,
                                const std::vector<int32_t>& seg_off, f2m_ctx** out) {
  if (!out) return fail(nullptr, F2M_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  g_create_error.clear();
  if (!xy || !row_ptr || !col) return fail(nullptr, F2M_ERR_INVALID_ARG, "NULL input array");
  if (n < 4 || n >= (1 << 24)) return fail(nullptr, F2M_ERR_INVALID_ARG, "n must be in [4, 2^24)");
  f2m_params p;
  if (params) p = *params; else f2m_default_params(&p);
  if (check_params_internal(p) != F2M_OK) return F2M_ERR_INVALID_ARG;

  f2m_ctx* c = new (std::nothrow) f2m_ctx();
  if (!c) return fail(nullptr, F2M_ERR_OOM, "host allocation");
  c->n = n;
  c->p = p;
  c->st = (cudaStream_t)stream;
  c->seg_off = seg_off;
  c->fb_cur = p.frac_bits;
  f2m_status s = F2M_OK;
  int32_t* d_col = nullptr;
  do {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = dalloc(&c->d_rp, n + 1);
    if (e == cudaSuccess) e = dalloc(&c->d_xy, n);
    if (e == cudaSuccess) e = dalloc(&c->d_check, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_rp, row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDefault, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_xy, xy, sizeof(int2) * n, cudaMemcpyDefault, c->st);
    int32_t nnz_h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz_h, c->d_rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) { s = cuda_fail(nullptr, e, "create: upload"); break; }
    if (nnz_h < 3 * (int64_t)n) { s = fail(nullptr, F2M_ERR_INVALID_ARG, "row_ptr[n] < 3n: some node has degree below 3"); break; }
    c->nnz = nnz_h;
    e = reset_check(c);
    if (e == cudaSuccess) e = launch_check(c->d_xy, c->d_rp, nullptr, n, c->nnz, c->d_check, c->st);
    CheckCtl h{};
    if (e == cudaSuccess) e = read_check(c, &h);
    if (e != cudaSuccess) { s = cuda_fail(nullptr, e, "create: check row_ptr"); break; }
    if (h.flags) { s = fail(nullptr, F2M_ERR_INVALID_ARG, check_message(h.flags, h.first_bad)); break; }
    e = dalloc(&d_col, c->nnz);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_col, col, sizeof(int32_t) * c->nnz, cudaMemcpyDefault, c->st);
    if (e == cudaSuccess) e = reset_check(c);
    if (e == cudaSuccess) e = launch_check(c->d_xy, c->d_rp, d_col, n, c->nnz, c->d_check, c->st);
    if (e == cudaSuccess) e = read_check(c, &h);
    if (e != cudaSuccess) { s = cuda_fail(nullptr, e, "create: check rows"); break; }
    if (h.flags) { s = fail(nullptr, F2M_ERR_INVALID_ARG, check_message(h.flags, h.first_bad)); break; }
    c->ec_cap = c->nnz + (c->nnz >> 3) + 4096;
    e = dalloc(&c->d_ec, c->ec_cap);
    if (e == cudaSuccess) e = launch_build_ec(c->d_xy, c->d_rp, d_col, n, c->d_ec, c->st);
    if (e == cudaSuccess) e = plan_renumber(c->d_xy, n, c->seg_off, c->plan, c->st);
    if (e == cudaSuccess)
      e = plan_build(c->d_rp, c->d_ec, n, c->nnz, c->num_sms, !(p.flags & F2M_FLAG_STREAMING_GDP),
                     p.frac_bits, p.gdp_ctas_per_sm, c->plan, c->st);
    if (e == cudaSuccess && seg_off.size() == 2 && !(p.flags & F2M_FLAG_ONE_SWEEP_GDP))
      e = plan_build2(c->plan, p.frac_bits, c->st);
    if (e == cudaSuccess && p.finisher) {
      e = alloc_finisher_buffers(c, c->ec_cap);
      c->fin_work = finisher_work_new();
      finisher_work_reserve(c->fin_work, n);
    }
    if (e == cudaSuccess) e = dalloc(&c->d_x2, c->ec_cap);
    c->x2_cap = c->ec_cap;
    // the pricing scan's and the merge's buffers, so that a solve allocates
    // nothing unless its graph outgrows them
    if (e == cudaSuccess && p.pricing) {
      c->pairs_cap = p.pricing_cap;
      c->tmp_col_cap = c->ec_cap;
      c->ec_alt_cap = c->ec_cap;
      e = dalloc(&c->d_ec_alt, c->ec_alt_cap);
      if (e == cudaSuccess) e = dalloc(&c->d_pts, n);
      if (e == cudaSuccess) e = dalloc(&c->d_count, 1);
      if (e == cudaSuccess) e = dalloc(&c->d_tile, 1);
      if (e == cudaSuccess) e = dalloc(&c->d_pairs, c->pairs_cap);
      if (e == cudaSuccess) e = dalloc(&c->d_deg, n + 1);
      if (e == cudaSuccess) e = dalloc(&c->d_tmp_rp, n + 1);
      if (e == cudaSuccess) e = dalloc(&c->d_new_rp, n + 1);
      if (e == cudaSuccess) e = dalloc(&c->d_block_sums, (int64_t)scan_scratch_ints(n));
      if (e == cudaSuccess) e = dalloc(&c->d_tmp_col, c->tmp_col_cap);
      if (e == cudaSuccess && seg_off.size() == 2) {  // the certifying scan's rows (one instance)
        e = dalloc(&c->d_lam_ref, n);
        if (e == cudaSuccess) e = dalloc(&c->d_raised, n);
        if (e == cudaSuccess) e = dalloc(&c->d_pts_raised, n);
        if (e == cudaSuccess) e = dalloc(&c->d_nraised, 1);
      }
    }
    if (e == cudaSuccess) e = dalloc(&c->d_lam[0], n);
    if (e == cudaSuccess) e = dalloc(&c->d_lam[1], n);
    if (e == cudaSuccess) e = dalloc(&c->d_lam2, n);
    if (e == cudaSuccess) e = dalloc(&c->d_gdp, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_scalar, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_bad, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_lam[0], 0, sizeof(int32_t) * n, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_lam[1], 0, sizeof(int32_t) * n, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_x2, 0, c->ec_cap, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) { s = cuda_fail(nullptr, e, "create: device setup"); break; }
  } while (0);
  dfree(d_col);
  if (s != F2M_OK) {
    f2m_destroy(c);
    return s;
  }
  *out = c;
  return F2M_OK;
}

__global__ void f2m_range_kernel(const int32_t* lam, int32_t n, long long limit, CheckCtl* ctl) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const long long x = lam[v];
    if (x >= limit || x <= -limit) {
      atomicOr(&ctl->flags, 1);
      atomicMin(&ctl->first_bad, (int)v);
    }
  }
}

extern "C" f2m_status f2m_set_lambda(f2m_ctx* c, const int32_t* lambda, int32_t frac_bits) {
  if (!c || !lambda) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  const int32_t F = c->p.frac_bits;
  if (frac_bits != F && frac_bits != F + 1) return fail(c, F2M_ERR_INVALID_ARG, "frac_bits must be F or F+1");
  int32_t* dst = frac_bits == F ? c->d_lam[c->cur] : c->d_lam2;
  CK(c, cudaMemcpyAsync(dst, lambda, sizeof(int32_t) * c->n, cudaMemcpyDefault, c->st));
  CK(c, reset_check(c));
  const long long limit = frac_bits == F ? kLamLimit : 2 * kLamLimit;
  f2m_range_kernel<<<(c->n + 255) / 256, 256, 0, c->st>>>(dst, c->n, limit, c->d_check);
  count_launch();
  CK(c, cudaGetLastError());
  CheckCtl h{};
  CK(c, read_check(c, &h));
  if (h.flags) return fail(c, F2M_ERR_INVALID_ARG, "lambda out of range at node " + std::to_string(h.first_bad));
  c->fb_cur = frac_bits;
  c->lam_version += 1;
  return F2M_OK;
}

extern "C" f2m_status f2m_set_degrees(f2m_ctx* c, const int32_t* b) {
  if (!c) return fail(c, F2M_ERR_INVALID_ARG, "NULL context");
  if (c->seg_off.size() != 2) return fail(c, F2M_ERR_INVALID_ARG, "degree requirements apply to a single-instance context");
  if (cut_count(c)) return fail(c, F2M_ERR_INVALID_ARG, "subtour cuts need b_v = 2");
  if (!b) {
    dfree(c->d_b);
    dfree(c->d_b_int);
    c->b_max = 2;
    return F2M_OK;
  }
  int32_t* d = nullptr;
  CK(c, dalloc(&d, c->n));
  cudaError_t e = cudaMemcpyAsync(d, b, sizeof(int32_t) * c->n, cudaMemcpyDefault, c->st);
  if (e == cudaSuccess) e = reset_check(c);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bad, 0, sizeof(unsigned long long), c->st);
  if (e == cudaSuccess) e = launch_check_degrees(c->d_rp, d, c->n, c->d_check, c->d_bad, c->st);
  unsigned long long bmax = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bmax, c->d_bad, sizeof(bmax), cudaMemcpyDeviceToHost, c->st);
  CheckCtl h{};
  if (e == cudaSuccess) e = read_check(c, &h);
  if (e != cudaSuccess) { dfree(d); return cuda_fail(c, e, "set_degrees"); }
  if (h.flags) { dfree(d); return fail(c, F2M_ERR_INVALID_ARG, check_message(h.flags, h.first_bad)); }
  int32_t* di = nullptr;  // the same in the renumbered order of the tiled kernel
  CK(c, dalloc(&di, c->n));
  e = gather_perm(d, c->plan.perm, c->n, di, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) { dfree(d); dfree(di); return cuda_fail(c, e, "set_degrees"); }
  dfree(c->d_b);
  dfree(c->d_b_int);
  c->d_b = d;
  c->d_b_int = di;
  c->b_max = (int32_t)bmax;
  return F2M_OK;
}

extern "C" f2m_status f2m_get_colors(f2m_ctx* c, int32_t* color, int32_t* ncolors) {
  if (!c) return fail(c, F2M_ERR_INVALID_ARG, "NULL context");
  if (c->classes.version != c->plan.version) {
    CK(c, color_classes(c->d_rp, c->d_ec, c->n, c->classes, c->st));
    c->classes.version = c->plan.version;
  }
  if (color) {
    CK(c, cudaMemcpyAsync(color, c->classes.color, sizeof(int32_t) * c->n, cudaMemcpyDefault, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  if (ncolors) *ncolors = c->classes.ncolors;
  return F2M_OK;
}

// lambda (device) and its fractional bits
const int32_t* f2m::cur_lambda(f2m_ctx* c, int32_t* fb) {
  *fb = c->fb_cur;
  return c->fb_cur == c->p.frac_bits ? c->d_lam[c->cur] : c->d_lam2;
}

f2m_status f2m::gdp_phase(f2m_ctx* c, int64_t max_sweeps, int64_t* sweeps, bool want_trace,
                            int64_t trace_cap, double* ms) {
  const int32_t F = c->p.frac_bits;
  c->lam_version += 1;
  if (c->fb_cur != F) {  // continue from the finisher's lambda: floor to F bits
    CK(c, launch_halve(c->d_lam2, c->d_lam[c->cur], c->n, c->st));
    c->fb_cur = F;
  }
  if (want_trace && trace_cap > c->trace_cap) {
    dfree(c->d_trace_b2);
    dfree(c->d_trace_ch);
    CK(c, dalloc(&c->d_trace_b2, trace_cap));
    CK(c, dalloc(&c->d_trace_ch, trace_cap));
    c->trace_cap = trace_cap;
  }
  long long* tb = want_trace ? c->d_trace_b2 : nullptr;
  unsigned long long* tc = want_trace ? reinterpret_cast<unsigned long long*>(c->d_trace_ch) : nullptr;
  const int64_t tcap = want_trace ? trace_cap : 0;
  if (cut_count(c) > 0) return cut_gdp_phase(c, max_sweeps, sweeps, tb, tc, tcap, ms);
  if (c->p.flags & F2M_FLAG_CLASS_SWEEPS) {
    CK(c, cudaEventRecord(c->ev0, c->st));
    if (c->classes.version != c->plan.version) {  // colour the graph held now
      CK(c, color_classes(c->d_rp, c->d_ec, c->n, c->classes, c->st));
      c->classes.version = c->plan.version;
    }
    CK(c, cudaMemsetAsync(c->d_gdp, 0, sizeof(GdpCtl), c->st));
    c->gdp_kernel = F2M_GDP_KERNEL_CLASSES;
    CK(c, launch_gdp_classes(c->d_rp, c->d_ec, c->d_b, c->b_max, c->d_lam[c->cur], c->classes, c->n,
                             F, c->p.damping_shift, max_sweeps, c->d_gdp, tb, tc, tcap,
                             c->p.barrier_budget_cycles, c->num_sms, c->st));
    CK(c, cudaEventRecord(c->ev1, c->st));
    GdpCtl h{};
    CK(c, cudaMemcpyAsync(&h, c->d_gdp, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (ms) *ms += elapsed_ms(c);
    *sweeps = h.sweeps;
    if (h.status & kGdpTimeout) return fail(c, F2M_ERR_TIMEOUT, "device-wide barrier wait exceeded its budget");
    if (h.status & kGdpOverflow) return fail(c, F2M_ERR_OVERFLOW, "|lambda| reached 2^29");
    return h.fixed_point ? F2M_OK : F2M_ERR_NOT_CONVERGED;
  }
  if (c->plan1_pending) {
    CK(c, plan_build_tiles(c->num_sms, c->p.frac_bits, c->p.gdp_ctas_per_sm, c->plan, c->st));
    c->plan1_pending = false;
  }
  if (c->plan2_pending) {
    CK(c, plan_build2(c->plan, c->p.frac_bits, c->st));
    c->plan2_pending = false;
  }
  CK(c, cudaMemsetAsync(c->d_gdp, 0, sizeof(GdpCtl), c->st));
  CK(c, cudaEventRecord(c->ev0, c->st));
  // degree requirements run on the two-sweep kernel or the streaming one (the
  // one-sweep tiled kernel holds Eq. 10's top-3 only)
  bool two = c->plan.valid2;  // two sweeps per barrier
  bool tiled = c->plan.valid && !c->d_b;
  if (two) {
    cudaError_t e = launch_gdp_tiled2(c->plan, c->d_lam[c->cur], c->p.damping_shift, max_sweeps, c->d_gdp, tb,
                                      tc, tcap, c->p.barrier_budget_cycles, c->d_b_int, c->b_max, c->st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
      cudaGetLastError();
      two = false;
    } else {
      CK(c, e);
    }
  }
  if (!two && tiled) {
    cudaError_t e = launch_gdp_tiled(c->plan, c->d_lam[c->cur], c->p.damping_shift, max_sweeps,
                                     c->d_gdp, tb, tc, tcap, c->p.barrier_budget_cycles, c->st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
      cudaGetLastError();
      tiled = false;  // the tiles do not fit on this device now: streaming kernel
    } else {
      CK(c, e);
    }
  }
  if (!two && !tiled)
    CK(c, launch_gdp(c->d_rp, c->d_ec, c->d_b, c->b_max, c->d_lam[c->cur], c->d_lam[c->cur ^ 1], c->n, F,
                     c->p.damping_shift, max_sweeps, c->d_gdp, tb, tc, tcap,
                     c->p.barrier_budget_cycles, c->num_sms, c->st));
  CK(c, cudaEventRecord(c->ev1, c->st));
  c->gdp_kernel = two ? (c->plan.packed2 ? F2M_GDP_KERNEL_TWO_SWEEP_PACKED : F2M_GDP_KERNEL_TWO_SWEEP)
                      : (tiled ? F2M_GDP_KERNEL_TILED : F2M_GDP_KERNEL_STREAMING);
  GdpCtl h{};
  CK(c, cudaMemcpyAsync(&h, c->d_gdp, sizeof(h), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (ms) *ms += elapsed_ms(c);
  if (two && !(h.status & kGdpTimeout)) {
    CK(c, plan_scatter_lambda(c->plan, (int)h.pad1, c->d_lam[c->cur], c->st));
    if (h.status & kGdpOddOverflow) {
      // the second sweep of a round overflowed: replay that round from its
      // input with the one-sweep kernel, which leaves lambda at the input of
      // the overflowing sweep
      const long long base = h.sweeps - 2;
      CK(c, cudaMemsetAsync(c->d_gdp, 0, sizeof(GdpCtl), c->st));
      GdpCtl h2{};
      if (c->d_b) {  // with degree requirements: the streaming kernel replays the round
        CK(c, launch_gdp(c->d_rp, c->d_ec, c->d_b, c->b_max, c->d_lam[c->cur], c->d_lam[c->cur ^ 1], c->n, F,
                         c->p.damping_shift, 2, c->d_gdp, tb ? tb + base : nullptr, tc ? tc + base : nullptr,
                         tcap > base ? tcap - base : 0, c->p.barrier_budget_cycles, c->num_sms, c->st));
        CK(c, cudaMemcpyAsync(&h2, c->d_gdp, sizeof(h2), cudaMemcpyDeviceToHost, c->st));
        CK(c, cudaStreamSynchronize(c->st));
        const bool ovf2 = (h2.status & kGdpOverflow) != 0;
        if (!(h2.status & kGdpTimeout) && ((ovf2 ? h2.sweeps - 1 : h2.sweeps) & 1)) c->cur ^= 1;
      } else {
        CK(c, launch_gdp_tiled(c->plan, c->d_lam[c->cur], c->p.damping_shift, 2, c->d_gdp,
                               tb ? tb + base : nullptr, tc ? tc + base : nullptr,
                               tcap > base ? tcap - base : 0, c->p.barrier_budget_cycles, c->st));
        CK(c, cudaMemcpyAsync(&h2, c->d_gdp, sizeof(h2), cudaMemcpyDeviceToHost, c->st));
        CK(c, cudaStreamSynchronize(c->st));
        const bool ovf2 = (h2.status & kGdpOverflow) != 0;
        if (!(h2.status & kGdpTimeout))
          CK(c, plan_scatter_lambda(c->plan, (int)((ovf2 ? h2.sweeps - 1 : h2.sweeps) % 3), c->d_lam[c->cur], c->st));
      }
      h.status = (h.status & ~kGdpOddOverflow) | h2.status;
      h.sweeps = base + h2.sweeps;
      h.fixed_point = h2.fixed_point;
    }
  }
  *sweeps = h.sweeps;
  const bool ovf = (h.status & kGdpOverflow) != 0;
  // the sweep that overflowed leaves lambda at its input; otherwise the last output
  const long long used = ovf ? h.sweeps - 1 : h.sweeps;
  if (!two && tiled) {
    if (!(h.status & kGdpTimeout))
      CK(c, plan_scatter_lambda(c->plan, (int)(used % 3), c->d_lam[c->cur], c->st));
  } else if (!two && (used & 1)) {
    c->cur ^= 1;
  }
  if (h.status & kGdpTimeout) return fail(c, F2M_ERR_TIMEOUT, "device-wide barrier wait exceeded its budget");
  if (ovf) return fail(c, F2M_ERR_OVERFLOW, "|lambda| reached 2^29");
  if (!h.fixed_point) return F2M_ERR_NOT_CONVERGED;
  return F2M_OK;
}

extern "C" f2m_status f2m_gdp(f2m_ctx* c, int64_t max_sweeps, int64_t* sweeps, int64_t* trace_bound2,
                              int64_t* trace_changed, int64_t trace_cap) {
  if (!c || max_sweeps < 0) return fail(c, F2M_ERR_INVALID_ARG, "bad argument");
  int64_t sw = 0;
  const bool want = trace_cap > 0 && (trace_bound2 || trace_changed);
  f2m_status s = gdp_phase(c, max_sweeps, &sw, want, trace_cap, nullptr);
  if (sweeps) *sweeps = sw;
  if (want && (s == F2M_OK || s == F2M_ERR_NOT_CONVERGED || s == F2M_ERR_OVERFLOW)) {
    const int64_t k = sw < trace_cap ? sw : trace_cap;
    if (k > 0 && trace_bound2)
      CK(c, cudaMemcpyAsync(trace_bound2, c->d_trace_b2, sizeof(int64_t) * k, cudaMemcpyDefault, c->st));
    if (k > 0 && trace_changed)
      CK(c, cudaMemcpyAsync(trace_changed, c->d_trace_ch, sizeof(int64_t) * k, cudaMemcpyDefault, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return s;
}

// pricing scan into d_pairs (grown until every pair fits); count in c->npairs
// Tile pairs of the pair triangle of every segment selected for this scan.
static void build_tiles(const f2m_ctx* c, std::vector<int4>& tiles) {
  tiles.clear();
  const int32_t nseg = (int32_t)c->seg_off.size() - 1;
  for (int32_t s = 0; s < nseg; ++s) {
    if (!c->seg_scan.empty() && !c->seg_scan[s]) continue;
    const int32_t a = c->seg_off[s], b = c->seg_off[s + 1];
    for (int32_t i0 = a; i0 < b; i0 += kPricingTile)
      for (int32_t j0 = i0; j0 < b; j0 += kPricingJ)  // half-height tiles: a shorter last wave
        tiles.push_back(make_int4(i0, i0 + kPricingTile < b ? i0 + kPricingTile : b, j0,
                                  j0 + kPricingJ < b ? j0 + kPricingJ : b));
  }
}

// the tensor-core scan's tile pairs: per scanned segment, i-blocks of
// kMmaTileI positions from its start, each against j-blocks of kMmaTileJ from
// the i-block's start (every pair u < v of the segment in exactly one)
// (tiles {i0, i1, j0, j1}; tblk {i-block, j-block, second j-block or -1};
// ranges: the blocks of kMmaTileI positions; a j-block pair starts on a block)
static void build_mma_tiles(const f2m_ctx* c, std::vector<int4>& tiles, std::vector<int4>& tblk,
                            std::vector<int2>& ranges) {
  static_assert(kMmaTileJ == kMmaTileI, "a j-block is a block");
  tiles.clear();
  tblk.clear();
  ranges.clear();
  const int32_t nseg = (int32_t)c->seg_off.size() - 1;
  for (int32_t s = 0; s < nseg; ++s) {
    if (!c->seg_scan.empty() && !c->seg_scan[s]) continue;
    const int32_t a = c->seg_off[s], b = c->seg_off[s + 1];
    const int32_t base = (int32_t)ranges.size();
    for (int32_t i0 = a; i0 < b; i0 += kMmaTileI) ranges.push_back(make_int2(i0, std::min(i0 + kMmaTileI, b)));
    for (int32_t i0 = a; i0 < b; i0 += kMmaTileI)
      for (int32_t j0 = i0; j0 < b; j0 += kMmaTileJ) {
        const int32_t jb = base + (j0 - a) / kMmaTileI;
        tiles.push_back(make_int4(i0, std::min(i0 + kMmaTileI, b), j0, std::min(j0 + kMmaTileJ, b)));
        tblk.push_back(make_int4(base + (i0 - a) / kMmaTileI, jb, -1, 0));
      }
  }
}

// pricing scan into d_pairs (grown until every pair fits); count in c->npairs,
// per-segment counts in c->seg_pairs
f2m_status f2m::price_internal(f2m_ctx* c, double* ms, const int32_t* lam_override) {
  if (!c->d_pts) {
    CK(c, dalloc(&c->d_pts, c->n));
    CK(c, dalloc(&c->d_count, 1));
    CK(c, dalloc(&c->d_tile, 1));
  }
  if (!c->d_pairs) {
    c->pairs_cap = c->p.pricing_cap;
    CK(c, dalloc(&c->d_pairs, c->pairs_cap));
  }
  int32_t fb = 0;
  const int32_t* lam = cur_lambda(c, &fb);
  if (lam_override) lam = lam_override;
  const int32_t nseg = (int32_t)c->seg_off.size() - 1;
  const bool plain = !lam_override && !cut_count(c);  // a scan of lambda itself, F2M terms only
  // The scan that certifies the finisher's lambda.  A complete scan at lambda
  // lam_ref left z >= 0 on every pair outside the CSR (the pairs it found were
  // merged); the finisher is the only change of lambda since, and returns
  // lambda' = lam_ref * 2^(fb - ref_fb) + delta.  Then z'_uv = z_uv 2^(fb -
  // ref_fb) - delta_u - delta_v can be negative only if delta_u > 0 or
  // delta_v > 0: only the rows of the nodes whose lambda rose are scanned,
  // against all points, for the same pairs as a full scan.
  if (plain && nseg == 1 && c->p.pricing == 1 && !(c->p.flags & F2M_FLAG_PRICING_TENSOR) && c->d_lam_ref &&
      c->ref_version == c->fin_src_version && c->lam_version == c->fin_dst_version && fb > c->ref_fb) {
    CK(c, cudaEventRecord(c->ev0, c->st));
    CK(c, launch_pricing_prep(c->d_xy, lam, nullptr, c->n, fb, c->d_pts, c->st));
    CK(c, launch_pricing_raised(lam, c->d_lam_ref, c->n, fb - c->ref_fb, c->d_pts, c->d_raised, c->d_pts_raised,
                                c->d_nraised, c->st));
    unsigned int nu = 0;
    CK(c, cudaMemcpyAsync(&nu, c->d_nraised, sizeof(nu), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    const int64_t ntiles_r = (int64_t)((nu + kPricingTile - 1) / kPricingTile) * ((c->n + kPricingJ - 1) / kPricingJ);
    for (bool first = true;; first = false) {
      if (!first) CK(c, cudaEventRecord(c->ev0, c->st));
      CK(c, launch_pricing_scan(c->d_pts, c->d_xy, lam, c->d_rp, c->d_ec, c->n, fb, nullptr, (int32_t)ntiles_r,
                                c->d_pairs, c->pairs_cap, c->d_count, c->d_tile, c->num_sms, c->st,
                                c->d_pts_raised, c->d_raised, (int32_t)nu));
      CK(c, cudaEventRecord(c->ev1, c->st));
      unsigned long long cnt = 0;
      CK(c, cudaMemcpyAsync(&cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaStreamSynchronize(c->st));
      if (ms) *ms += elapsed_ms(c);
      c->npairs = (int64_t)cnt;
      if ((int64_t)cnt <= c->pairs_cap) break;
      dfree(c->d_pairs);
      c->pairs_cap = (int64_t)cnt + ((int64_t)cnt >> 2) + 1024;
      CK(c, dalloc(&c->d_pairs, c->pairs_cap));
    }
    c->seg_pairs.assign(1, c->npairs);
    c->last_scan_rows = (int64_t)nu;
    c->last_scan_pairs = (int64_t)nu * c->n;
    // a complete result for this lambda: it is the next reference
    CK(c, cudaMemcpyAsync(c->d_lam_ref, lam, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->st));
    c->ref_fb = fb;
    c->ref_version = c->lam_version;
    return F2M_OK;
  }
  c->last_scan_rows = -1;
  c->last_scan_pairs = 0;
  for (int32_t sg = 0; sg < nseg; ++sg)
    if (c->seg_scan.empty() || c->seg_scan[sg]) {
      const int64_t m = c->seg_off[sg + 1] - c->seg_off[sg];
      c->last_scan_pairs += m * (m - 1) / 2;
    }
  // full scan: with the fp32 filter (caller order), or on the tensor cores
  // (renumbered order); culled scan: fp32 filter in the renumbered (Morton)
  // order, so that a tile is a compact patch with a small bounding box
  const bool culled = c->p.pricing == 2;
  const bool mma = !culled && (c->p.flags & F2M_FLAG_PRICING_TENSOR);
  const int kind = mma ? 1 : 0;
  // the full scan's tile-pair list depends only on the segments scanned: it
  // stays on the device from one scan to the next while they are the same
  std::vector<int4> tiles;
  const bool reuse = !culled && c->tiles_valid && c->tiles_kind == kind && c->tiles_seg_scan == c->seg_scan &&
                     c->tiles_seg_off == c->seg_off;
  if (mma && !c->d_pts4) {
    CK(c, dalloc(&c->d_pts4, c->n));
    CK(c, dalloc(&c->d_pstat, 1));
    CK(c, dalloc(&c->d_mncand, 1));
    c->mcand_cap = std::max<int64_t>(4LL * c->n, 1 << 20);
    CK(c, dalloc(&c->d_mcand, c->mcand_cap));
  }
  if (!reuse) {
    if (mma) {
      std::vector<int4> tblk;
      std::vector<int2> ranges;
      build_mma_tiles(c, tiles, tblk, ranges);
      if ((int64_t)ranges.size() > c->mblocks_cap) {
        dfree(c->d_mranges);
        dfree(c->d_mbox);
        dfree(c->d_mlmax);
        c->mblocks_cap = (int64_t)ranges.size() + 64;
        CK(c, dalloc(&c->d_mranges, c->mblocks_cap));
        CK(c, dalloc(&c->d_mbox, c->mblocks_cap));
        CK(c, dalloc(&c->d_mlmax, c->mblocks_cap));
      }
      if ((int64_t)tblk.size() > c->mtiles_cap) {
        dfree(c->d_mtblk);
        dfree(c->d_mframes);
        c->mtiles_cap = (int64_t)tblk.size() + 64;
        CK(c, dalloc(&c->d_mtblk, c->mtiles_cap));
        CK(c, dalloc(&c->d_mframes, c->mtiles_cap));
      }
      if (!ranges.empty())
        CK(c, cudaMemcpyAsync(c->d_mranges, ranges.data(), sizeof(int2) * ranges.size(), cudaMemcpyHostToDevice,
                              c->st));
      if (!tblk.empty())
        CK(c, cudaMemcpyAsync(c->d_mtblk, tblk.data(), sizeof(int4) * tblk.size(), cudaMemcpyHostToDevice, c->st));
      c->mblocks = (int64_t)ranges.size();
    } else {
      build_tiles(c, tiles);
    }
  }
  CK(c, cudaEventRecord(c->ev0, c->st));
  if (mma)
    CK(c, launch_pricing_mma_prep(c->d_xy, lam, c->plan.perm, c->n, c->d_pts4, c->st));
  else
    CK(c, launch_pricing_prep(c->d_xy, lam, culled ? c->plan.perm : nullptr, c->n, fb, c->d_pts, c->st));
  if (culled && !tiles.empty()) {
    // A pair (u, v) can have z < 0 only if its distance is below s_u + s_v
    // (the filter's radii, see pricing.cu), so a tile pair whose bounding
    // boxes are at least max s + max s apart holds none: it is skipped.
    // the point ranges of the tiles: per segment, steps of kPricingTile from its start
    std::vector<int2> ranges;
    std::vector<int32_t> base(nseg + 1, 0);
    for (int32_t sg = 0; sg < nseg; ++sg) {
      base[sg] = (int32_t)ranges.size();
      for (int32_t i0 = c->seg_off[sg]; i0 < c->seg_off[sg + 1]; i0 += kPricingTile)
        ranges.push_back(make_int2(i0, std::min(i0 + kPricingTile, c->seg_off[sg + 1])));
    }
    auto range_id = [&](int32_t i0) {
      const int32_t sg = (int32_t)(std::upper_bound(c->seg_off.begin(), c->seg_off.end(), i0) - c->seg_off.begin()) - 1;
      return base[sg] + (i0 - c->seg_off[sg]) / kPricingTile;
    };
    std::vector<int32_t> rid_of(tiles.size()), cid_of(tiles.size());
    for (size_t k = 0; k < tiles.size(); ++k) {
      rid_of[k] = range_id(tiles[k].x);
      cid_of[k] = range_id(tiles[k].z);
    }
    if ((int64_t)ranges.size() > c->ranges_cap) {
      dfree(c->d_ranges);
      dfree(c->d_boxes);
      dfree(c->d_smax);
      c->ranges_cap = (int64_t)ranges.size() + 64;
      CK(c, dalloc(&c->d_ranges, c->ranges_cap));
      CK(c, dalloc(&c->d_boxes, c->ranges_cap));
      CK(c, dalloc(&c->d_smax, c->ranges_cap));
    }
    CK(c, cudaMemcpyAsync(c->d_ranges, ranges.data(), sizeof(int2) * ranges.size(), cudaMemcpyHostToDevice, c->st));
    CK(c, launch_pricing_boxes(c->d_pts, c->d_ranges, (int32_t)ranges.size(), c->d_boxes, c->d_smax, c->st));
    std::vector<float4> box(ranges.size());
    std::vector<float> smax(ranges.size());
    CK(c, cudaMemcpyAsync(box.data(), c->d_boxes, sizeof(float4) * box.size(), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaMemcpyAsync(smax.data(), c->d_smax, sizeof(float) * smax.size(), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    std::vector<int4> kept;
    kept.reserve(tiles.size());
    for (size_t k = 0; k < tiles.size(); ++k) {
      const float4 a = box[rid_of[k]], b = box[cid_of[k]];
      const double gx = std::max(0.0, std::max((double)a.x - b.z, (double)b.x - a.z));
      const double gy = std::max(0.0, std::max((double)a.y - b.w, (double)b.y - a.w));
      const double r = (double)smax[rid_of[k]] + (double)smax[cid_of[k]];
      if (gx * gx + gy * gy < r * r * (1.0 + 1e-9) + 1.0) kept.push_back(tiles[k]);
    }
    tiles.swap(kept);
  }
  if (!reuse) {
    if ((int64_t)tiles.size() > c->tiles_cap) {
      dfree(c->d_tiles);
      c->tiles_cap = (int64_t)tiles.size() + 64;
      CK(c, dalloc(&c->d_tiles, c->tiles_cap));
    }
    if (!tiles.empty())
      CK(c, cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, c->st));
    c->tiles_valid = !culled;
    c->tiles_kind = kind;
    c->tiles_seg_scan = c->seg_scan;
    c->tiles_seg_off = c->seg_off;
    c->ntiles = (int64_t)tiles.size();
  }
  const int64_t ntiles = c->ntiles;
  bool first = true;
  for (;;) {
    if (!first) CK(c, cudaEventRecord(c->ev0, c->st));
    first = false;
    if (mma)
      CK(c, launch_pricing_mma_scan(c->d_pts4, c->d_xy, lam, c->d_rp, c->d_ec, fb, c->d_tiles, c->d_mtblk,
                                    (int32_t)ntiles, c->d_mranges, (int32_t)c->mblocks, c->d_mbox, c->d_mlmax,
                                    c->d_mframes, c->d_mcand, c->mcand_cap, c->d_mncand, c->d_pairs,
                                    c->pairs_cap, c->d_count, c->d_tile, c->d_pstat, c->num_sms, c->st));
    else
      CK(c, launch_pricing_scan(c->d_pts, c->d_xy, lam, c->d_rp, c->d_ec, c->n, fb, c->d_tiles,
                                (int32_t)ntiles, c->d_pairs, c->pairs_cap, c->d_count, c->d_tile,
                                c->num_sms, c->st));
    CK(c, cudaEventRecord(c->ev1, c->st));
    unsigned long long cnt = 0;
    int32_t pstat = 0;
    unsigned long long ncand = 0;
    CK(c, cudaMemcpyAsync(&cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->st));
    if (mma) {
      CK(c, cudaMemcpyAsync(&pstat, c->d_pstat, sizeof(pstat), cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(&ncand, c->d_mncand, sizeof(ncand), cudaMemcpyDeviceToHost, c->st));
    }
    CK(c, cudaStreamSynchronize(c->st));
    if (ms) *ms += elapsed_ms(c);
    if (pstat) return fail(c, F2M_ERR_TIMEOUT, "pricing scan: a tensor-core wait ran past its budget");
    if (mma && (int64_t)ncand > c->mcand_cap) {  // the candidate list overflowed: grow it, scan again
      dfree(c->d_mcand);
      c->mcand_cap = (int64_t)ncand + ((int64_t)ncand >> 2) + 1024;
      CK(c, dalloc(&c->d_mcand, c->mcand_cap));
      continue;
    }
    c->npairs = (int64_t)cnt;
    if ((int64_t)cnt <= c->pairs_cap) break;
    dfree(c->d_pairs);
    c->pairs_cap = (int64_t)cnt + ((int64_t)cnt >> 2) + 1024;
    CK(c, dalloc(&c->d_pairs, c->pairs_cap));
  }
  if (plain && c->d_lam_ref) {  // the reference of a later certifying scan
    CK(c, cudaMemcpyAsync(c->d_lam_ref, lam, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->st));
    c->ref_fb = fb;
    c->ref_version = c->lam_version;
  }
  c->seg_pairs.assign(nseg, 0);
  if (nseg == 1) {
    c->seg_pairs[0] = c->npairs;
  } else if (c->npairs > 0) {
    std::vector<int2> h(c->npairs);
    CK(c, cudaMemcpyAsync(h.data(), c->d_pairs, sizeof(int2) * c->npairs, cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    for (const int2& q : h) {
      const int32_t s = (int32_t)(std::upper_bound(c->seg_off.begin(), c->seg_off.end(), q.x) -
                                  c->seg_off.begin()) - 1;
      c->seg_pairs[s] += 1;
    }
  }
  return F2M_OK;
}

extern "C" f2m_status f2m_pricing_mma_check(int64_t rounds, uint64_t seed, int64_t* checked,
                                            int64_t* mismatches) {
  if (!checked || !mismatches || rounds < 0) return fail(nullptr, F2M_ERR_INVALID_ARG, "bad argument");
  unsigned long long* d = nullptr;
  cudaError_t e = dalloc(&d, 3);
  if (e == cudaSuccess) e = cudaMemset(d, 0, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = launch_pricing_mma_check(rounds, seed, d, d + 1, reinterpret_cast<int32_t*>(d + 2), nullptr);
  unsigned long long h[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (d) dev_free_synced(d);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_pricing_mma_check");
  *checked = (int64_t)h[0];
  *mismatches = (int64_t)h[1];
  if ((int32_t)h[2]) return fail(nullptr, F2M_ERR_TIMEOUT, "f2m_pricing_mma_check: an mbarrier wait gave up");
  return F2M_OK;
}

extern "C" f2m_status f2m_price(f2m_ctx* c, int64_t* count, int32_t* pairs, int64_t cap) {
  if (!c || !count) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  f2m_status s = cut_count(c) ? cut_price(c, nullptr) : price_internal(c, nullptr);
  if (s != F2M_OK) return s;
  *count = c->npairs;
  if (pairs && c->npairs > 0 && c->npairs <= cap) {
    CK(c, cudaMemcpyAsync(pairs, c->d_pairs, sizeof(int2) * c->npairs, cudaMemcpyDefault, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return F2M_OK;
}

// CSR u pairs (device array of npairs int2)
f2m_status f2m::merge_internal(f2m_ctx* c, const int2* d_pairs, int64_t npairs, double* ms) {
  const int32_t n = c->n;
  if (!c->d_deg) {
    CK(c, dalloc(&c->d_deg, n + 1));
    CK(c, dalloc(&c->d_tmp_rp, n + 1));
    CK(c, dalloc(&c->d_new_rp, n + 1));
    CK(c, dalloc(&c->d_block_sums, (int64_t)scan_scratch_ints(n)));
  }
  const int64_t need = c->nnz + 2 * npairs;
  if (need >= INT_MAX) return fail(c, F2M_ERR_INVALID_ARG, "graph would exceed 2^31 entries");
  if (need > c->tmp_col_cap) {
    dfree(c->d_tmp_col);
    c->tmp_col_cap = need + (need >> 3);
    CK(c, dalloc(&c->d_tmp_col, c->tmp_col_cap));
  }
  MergeBuffers mb{c->d_deg, c->d_tmp_rp, c->d_tmp_col, c->d_new_rp, c->d_block_sums, c->d_check};
  CK(c, reset_check(c));
  CK(c, cudaEventRecord(c->ev0, c->st));
  CK(c, launch_merge_count(c->d_rp, d_pairs, npairs, n, mb, c->st));
  CK(c, launch_merge_fill(c->d_rp, c->d_ec, d_pairs, npairs, n, mb, c->st));
  if (need > c->ec_alt_cap) {  // the array the merged rows go to
    dfree(c->d_ec_alt);
    c->ec_alt_cap = need + (need >> 3);
    CK(c, dalloc(&c->d_ec_alt, c->ec_alt_cap));
  }
  if (need > c->x2_cap) {
    dfree(c->d_x2);
    c->x2_cap = need + (need >> 3);
    CK(c, dalloc(&c->d_x2, c->x2_cap));
  }
  CK(c, launch_merge_finish(c->d_xy, c->d_rp, c->d_ec, n, mb, c->d_ec_alt, c->st));
  std::swap(c->d_ec, c->d_ec_alt);
  std::swap(c->ec_cap, c->ec_alt_cap);
  CK(c, cudaMemcpyAsync(c->d_rp, c->d_new_rp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice, c->st));
  int32_t nnz_h = 0;
  CK(c, cudaMemcpyAsync(&nnz_h, c->d_new_rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CheckCtl h{};
  CK(c, read_check(c, &h));
  c->nnz = nnz_h;
  if (h.flags) return fail(c, F2M_ERR_INVALID_ARG, check_message(h.flags, h.first_bad));
  // the internal CSR now (the finisher reads it); the tiles of the
  // shared-memory GDP kernels only serve GDP phases: built when the next one
  // starts (a merge before the finisher and the last scan needs none)
  CK(c, plan_build(c->d_rp, c->d_ec, n, c->nnz, c->num_sms, false, c->p.frac_bits, c->p.gdp_ctas_per_sm,
                   c->plan, c->st));
  c->plan1_pending = c->seg_off.size() == 2 && !(c->p.flags & F2M_FLAG_STREAMING_GDP);
  c->plan.valid2 = false;
  c->plan2_pending = c->seg_off.size() == 2 && !(c->p.flags & F2M_FLAG_ONE_SWEEP_GDP);
  CK(c, cudaEventRecord(c->ev1, c->st));
  if (ms) *ms += elapsed_ms(c);
  return F2M_OK;
}

extern "C" f2m_status f2m_add_edges(f2m_ctx* c, const int32_t* pairs, int64_t npairs) {
  if (!c || (npairs > 0 && !pairs) || npairs < 0) return fail(c, F2M_ERR_INVALID_ARG, "bad argument");
  if (npairs == 0) return F2M_OK;
  int2* d = nullptr;
  CK(c, dalloc(&d, npairs));
  cudaError_t e = cudaMemcpyAsync(d, pairs, sizeof(int2) * npairs, cudaMemcpyDefault, c->st);
  if (e != cudaSuccess) { dfree(d); return cuda_fail(c, e, "add_edges: upload"); }
  f2m_status s = merge_internal(c, d, npairs, nullptr);
  cudaStreamSynchronize(c->st);
  dfree(d);
  return s;
}

f2m_status f2m::extract_internal(f2m_ctx* c, int64_t* bad, double* ms) {
  if (cut_count(c)) return cut_bound_extract(c, true, nullptr, bad);
  int32_t fb = 0;
  const int32_t* lam = cur_lambda(c, &fb);
  CK(c, cudaEventRecord(c->ev0, c->st));
  CK(c, launch_extract(c->d_rp, c->d_ec, c->d_b, lam, c->n, fb, c->d_x2, c->d_bad, c->st));
  CK(c, cudaEventRecord(c->ev1, c->st));
  unsigned long long b = 0;
  CK(c, cudaMemcpyAsync(&b, c->d_bad, sizeof(b), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (ms) *ms += elapsed_ms(c);
  *bad = (int64_t)b;
  return F2M_OK;
}

extern "C" f2m_status f2m_extract(f2m_ctx* c, uint8_t* x2, int64_t* bad) {
  if (!c || !bad) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  f2m_status s = extract_internal(c, bad, nullptr);
  if (s != F2M_OK) return s;
  if (x2) {
    CK(c, cudaMemcpyAsync(x2, c->d_x2, c->nnz, cudaMemcpyDefault, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return F2M_OK;
}

f2m_status f2m::bound_internal(f2m_ctx* c, int64_t* b2) {
  if (cut_count(c)) return cut_bound_extract(c, false, b2, nullptr);
  int32_t fb = 0;
  const int32_t* lam = cur_lambda(c, &fb);
  CK(c, launch_bound(c->d_rp, c->d_ec, c->d_b, lam, c->n, fb, c->d_scalar, c->st));
  long long h = 0;
  CK(c, cudaMemcpyAsync(&h, c->d_scalar, sizeof(h), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  *b2 = h;
  return F2M_OK;
}

// Phase 1 of the finisher on the GPU for the given blocks (internal node
// ranges): the state it leaves is in d_fy (flow), d_fpi and d_fex.
static f2m_status fin_gpu_phase1(f2m_ctx* c, const std::vector<int2>& fblocks, const int32_t* d_exl,
                                 const int32_t* d_lam_int, const unsigned long long* missing,
                                 int64_t* pushes_out) {
  const int32_t n = c->n;
  const int32_t nb = (int32_t)fblocks.size();
  GdpPlan& P = c->plan;
  if (!c->d_fpi) {  // node-sized state, both copies of every node
    CK(c, dalloc(&c->d_fpi, 2LL * n));
    CK(c, dalloc(&c->d_fdist, 2LL * n));
    CK(c, dalloc(&c->d_fex, 2LL * n));
    CK(c, dalloc(&c->d_fvia, 2LL * n));
    CK(c, dalloc(&c->d_fpred, 2LL * n));
    CK(c, dalloc(&c->d_freach, 2LL * n));
    CK(c, dalloc(&c->d_fclos, 2LL * n));
    CK(c, dalloc(&c->d_forder, 2LL * n));
    CK(c, dalloc(&c->d_fstat, 1));
    CK(c, pin_alloc((void**)&c->h_fpi, sizeof(int64_t) * 2 * (size_t)n));
    CK(c, pin_alloc((void**)&c->h_fex, sizeof(int32_t) * 2 * (size_t)n));
  }
  if (nb > c->fblk_cap) {
    dfree(c->d_fblk);
    dfree(c->d_fcaps);
    dfree(c->d_fheap_off);
    dfree(c->d_fpush);
    c->fblk_cap = nb + nb / 4 + 16;
    CK(c, dalloc(&c->d_fblk, c->fblk_cap));
    CK(c, dalloc(&c->d_fcaps, c->fblk_cap));
    CK(c, dalloc(&c->d_fheap_off, c->fblk_cap + 1));
    CK(c, dalloc(&c->d_fpush, c->fblk_cap));
  }
  CK(c, cudaMemcpyAsync(c->d_fblk, fblocks.data(), sizeof(int2) * nb, cudaMemcpyHostToDevice, c->st));
  CK(c, launch_fin_block_caps(c->d_fblk, nb, P.irp, c->d_fcaps, c->st));
  std::vector<long long> caps(nb), off(nb + 1, 0);
  CK(c, cudaMemcpyAsync(caps.data(), c->d_fcaps, sizeof(long long) * nb, cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  // every twin entry must exist before the kernel follows them
  if (*missing) return fail(c, F2M_ERR_INVALID_ARG, "finisher: CSR not symmetric");
  for (int32_t k = 0; k < nb; ++k) off[k + 1] = off[k] + caps[k];
  const size_t item = fin_heap_item_bytes();
  if ((int64_t)off[nb] > c->fheap_cap) {
    dfree(c->d_fheap);
    c->fheap_cap = off[nb] + off[nb] / 4 + 1024;
    CK(c, dalloc(&c->d_fheap, (int64_t)(c->fheap_cap * item)));
  }
  CK(c, cudaMemcpyAsync(c->d_fheap_off, off.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice, c->st));
  CK(c, cudaMemsetAsync(c->d_fstat, 0, sizeof(int32_t), c->st));
  CK(c, launch_fin_blocks(n, c->d_fblk, nb, P.irp, P.iec, c->d_twin, c->d_fy, d_exl, d_lam_int, c->p.frac_bits,
                          c->d_fpi, c->d_fdist, c->d_fex, c->d_fvia, c->d_fpred, c->d_freach, c->d_fclos,
                          c->d_fheap, c->d_fheap_off, c->d_forder, c->d_fpush, c->d_fstat,
                          4 * c->p.barrier_budget_cycles, c->st));
  std::vector<long long> pushes(nb);
  int32_t stat = 0;
  CK(c, cudaMemcpyAsync(pushes.data(), c->d_fpush, sizeof(long long) * nb, cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaMemcpyAsync(&stat, c->d_fstat, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (stat) return fail(c, F2M_ERR_TIMEOUT, "finisher phase 1 on the GPU ran past its budget or its heap");
  int64_t tot = 0;
  for (long long q : pushes) tot += q;
  *pushes_out = tot;
  c->fin_stats.aug[0] += tot;
  c->fin_stats.phase1_gpu = 1;
  return F2M_OK;
}

// Exact finisher: device prep (twin arcs, initial flow, surpluses) on the
// renumbered CSR, successive shortest paths on the host (phase 1 on the GPU
// with F2M_FLAG_FINISHER_GPU), results scattered back to caller order on the
// device.
f2m_status f2m::finisher_internal(f2m_ctx* c, int64_t* aug, const uint8_t* h_include) {
  using clk = std::chrono::steady_clock;
  const auto t_prep = clk::now();
  c->fin_src_version = c->lam_version;
  c->lam_version += 1;  // lambda changes below (or the call fails)
  c->fin_dst_version = h_include ? -3 : c->lam_version;  // a partial call does not qualify
  const int32_t n = c->n;
  const int32_t F = c->p.frac_bits;
  GdpPlan& P = c->plan;
  const int32_t nseg = (int32_t)c->seg_off.size() - 1;
  if (c->fin_cap < c->nnz) CK(c, alloc_finisher_buffers(c, c->ec_cap));
  if (!c->fin_work) c->fin_work = finisher_work_new();
  // the host mirror for this call; on any return the stream is drained
  // before the next call may take the mirror (no copy still reads or writes it)
  std::unique_lock<std::mutex> mirror_lock(g_mirror.mu);
  struct Drain {
    cudaStream_t st;
    ~Drain() { cudaStreamSynchronize(st); }
  } drain{c->st};
  CK(c, take_mirror(c));
  static const int32_t hw = (int32_t)std::thread::hardware_concurrency();
  unsigned long long missing = 0;
  const bool twin_new = c->twin_version != P.version;
  if (twin_new) {  // the graph changed: reverse entries again
    CK(c, cudaMemsetAsync(c->d_bad, 0, sizeof(unsigned long long), c->st));
    CK(c, fin_build_twin(P, c->d_twin, c->d_bad, c->st));
    CK(c, cudaMemcpyAsync(&missing, c->d_bad, sizeof(missing), cudaMemcpyDeviceToHost, c->st));
  }
  int32_t* d_lam_int = P.ilam[0];   // free outside a GDP phase
  int32_t* d_lam2_int = P.ilam[1];
  if (!c->d_exl) CK(c, dalloc(&c->d_exl, n));
  int32_t* d_exl = c->d_exl;
  CK(c, fin_prepare(P, c->d_lam[c->cur], c->d_b, F, d_lam_int, c->d_fy, d_exl, c->st));
  if (c->d_fin_include)
    CK(c, launch_batch_mask_surplus(d_exl, c->d_seg_off, nseg, c->d_fin_include, n, c->st));
  // phase 1 of the successive shortest paths on the GPU, one warp per block,
  // when the flags ask for it: it leaves the flow, potentials and surpluses of
  // the host's phase 1, and the host goes on with phases 2 and 3
  std::vector<int2> fblocks;
  for (int32_t sg = 0; sg < nseg; ++sg) {
    if (h_include && !h_include[sg]) continue;
    for (int32_t b0 = c->seg_off[sg]; b0 < c->seg_off[sg + 1]; b0 += kFinBlockNodes)
      fblocks.push_back(make_int2(b0, std::min(b0 + kFinBlockNodes, c->seg_off[sg + 1])));
  }
  const uint32_t fl = c->p.flags;
  const bool gpu1 = !fblocks.empty() && !(fl & F2M_FLAG_FINISHER_HOST) && (fl & F2M_FLAG_FINISHER_GPU);
  int64_t gpu_pushes = 0;
  double ms_gpu1 = 0;  // wall time of phase 1 on the GPU: phase 1's, not prep's
  if (gpu1) {
    const auto t1 = clk::now();
    const f2m_status s1 = fin_gpu_phase1(c, fblocks, d_exl, d_lam_int, &missing, &gpu_pushes);
    if (s1 != F2M_OK) return s1;
    ms_gpu1 = std::chrono::duration<double, std::milli>(clk::now() - t1).count();
    c->fin_stats.ms_phase[0] += ms_gpu1;
  }
  // the host copy of the graph: whole (cached per graph version), or, when a
  // batch names the instances the finisher works on, just theirs (node and
  // entry ranges of segments are contiguous in the internal order); the others
  // keep lambda, doubled to F+1 bits on the device
  std::vector<int2> ranges;   // entry ranges [x, y) that the host reads and writes
  std::vector<int2> nranges;  // their node ranges
  bool wide = false;          // one span that also covers instances the finisher leaves alone
  if (h_include) {
    CK(c, launch_double(d_lam_int, d_lam2_int, n, c->st));
    CK(c, cudaMemcpyAsync(c->h_irp, P.irp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    c->fin_version = -1;  // the host copy is partial from here on
    for (int32_t sg = 0; sg < nseg; ++sg) {
      if (!h_include[sg]) continue;
      const int32_t v0 = c->seg_off[sg], v1 = c->seg_off[sg + 1];
      const int32_t e0 = c->h_irp[v0], e1 = c->h_irp[v1];
      if (!nranges.empty() && nranges.back().y == v0) {
        nranges.back().y = v1;
        ranges.back().y = e1;
      } else {
        nranges.push_back(make_int2(v0, v1));
        ranges.push_back(make_int2(e0, e1));
      }
    }
    // many ranges: one span from the first to the last instead (the copies'
    // fixed cost dominates); the instances between are copied and written
    // back unchanged, their lambda at F+1 bits set on the host below
    if (ranges.size() > 8) {
      ranges.assign(1, make_int2(ranges.front().x, ranges.back().y));
      nranges.assign(1, make_int2(nranges.front().x, nranges.back().y));
      wide = true;
    }
    for (size_t k = 0; k < ranges.size(); ++k) {
      const int2 q = ranges[k], v = nranges[k];
      const size_t m = (size_t)(q.y - q.x), nv = (size_t)(v.y - v.x);
      CK(c, cudaMemcpyAsync(c->h_iec + q.x, P.iec + q.x, sizeof(int2) * m, cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_twin + q.x, c->d_twin + q.x, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_y + q.x, c->d_fy + q.x, m, cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_exl + v.x, d_exl + v.x, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_lam + v.x, d_lam_int + v.x, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost, c->st));
    }
  } else {
    CK(c, cudaMemcpyAsync(c->h_exl, d_exl, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaMemcpyAsync(c->h_lam, d_lam_int, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st));
    if (c->fin_version != P.version) {
      CK(c, cudaMemcpyAsync(c->h_irp, P.irp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_iec, P.iec, sizeof(int2) * c->nnz, cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_twin, c->d_twin, sizeof(int32_t) * c->nnz, cudaMemcpyDeviceToHost, c->st));
      c->fin_version = P.version;
    }
    CK(c, cudaMemcpyAsync(c->h_y, c->d_fy, c->nnz, cudaMemcpyDeviceToHost, c->st));
    ranges.push_back(make_int2(0, (int32_t)c->nnz));
    nranges.push_back(make_int2(0, n));
  }
  if (gpu1) {  // phase 1's potentials and surpluses, both copies of the nodes worked on
    for (const int2& v : nranges) {
      const size_t nv = (size_t)(v.y - v.x);
      CK(c, cudaMemcpyAsync(c->h_fpi + v.x, c->d_fpi + v.x, sizeof(int64_t) * nv, cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_fpi + n + v.x, c->d_fpi + n + v.x, sizeof(int64_t) * nv, cudaMemcpyDeviceToHost,
                            c->st));
      CK(c, cudaMemcpyAsync(c->h_fex + v.x, c->d_fex + v.x, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaMemcpyAsync(c->h_fex + n + v.x, c->d_fex + n + v.x, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost,
                            c->st));
    }
  }
  // the host's worker threads wake while the device prepares and copies
  finisher_pool_wake(std::min<int32_t>(hw, (int32_t)fblocks.size()));
  CK(c, cudaStreamSynchronize(c->st));
  if (twin_new) {
    if (missing) return fail(c, F2M_ERR_INVALID_ARG, "finisher: CSR not symmetric");
    c->twin_version = P.version;
  }
  c->fin_stats.ms_prep += std::chrono::duration<double, std::milli>(clk::now() - t_prep).count() - ms_gpu1;
  const int r = host_finisher(n, c->h_irp, c->h_iec, c->h_twin, c->h_y, c->h_exl, c->h_lam, F,
                              c->h_lam2, c->seg_off.data(), nseg, h_include, hw > 1 ? hw : 1, aug,
                              c->fin_work, &c->fin_stats, gpu1 ? c->h_fpi : nullptr, gpu1 ? c->h_fex : nullptr);
  *aug += gpu_pushes;
  const auto t_scatter = clk::now();
  if (r == 7)
    return fail(c, F2M_ERR_INFEASIBLE, c->d_b ? "no fractional b-matching exists on the candidate graph"
                                              : "no fractional 2-matching exists on the candidate graph");
  if (r == 5) return fail(c, F2M_ERR_OVERFLOW, "finisher lambda out of range");
  if (r != 0) return fail(c, F2M_ERR_INVALID_ARG, "finisher failed");
  if (wide) {  // the instances left alone inside the span keep lambda, doubled
    for (int32_t sg = 0; sg < nseg; ++sg) {
      if (h_include[sg] || c->seg_off[sg] < nranges[0].x || c->seg_off[sg + 1] > nranges[0].y) continue;
      for (int32_t v = c->seg_off[sg]; v < c->seg_off[sg + 1]; ++v) c->h_lam2[v] = 2 * c->h_lam[v];
    }
  }
  for (size_t k = 0; k < ranges.size(); ++k) {
    const int2 q = ranges[k], v = nranges[k];
    CK(c, cudaMemcpyAsync(c->d_fy + q.x, c->h_y + q.x, (size_t)(q.y - q.x), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(d_lam2_int + v.x, c->h_lam2 + v.x, sizeof(int32_t) * (size_t)(v.y - v.x),
                          cudaMemcpyHostToDevice, c->st));
  }
  CK(c, fin_scatter(P, c->d_rp, c->d_fy, c->d_twin, d_lam2_int, c->d_x2, c->d_lam2, c->d_seg_off,
                    (int32_t)c->seg_off.size() - 1, c->d_fin_include, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  c->fin_stats.ms_scatter += std::chrono::duration<double, std::milli>(clk::now() - t_scatter).count();
  c->fb_cur = F + 1;
  return F2M_OK;
}

void f2m::copy_finisher_stats(const f2m_ctx* c, f2m_info* info) {
  const FinisherStats& f = c->fin_stats;
  info->finish_phase1_gpu = f.phase1_gpu;
  info->ms_finish_prep = f.ms_prep;
  info->ms_finish_scatter = f.ms_scatter;
  for (int k = 0; k < 3; ++k) {
    info->ms_finish_phase[k] = f.ms_phase[k];
    info->finish_aug_phase[k] = f.aug[k];
  }
  info->finish_threads = f.threads;
}

// The solve loop; its decisions match the CPU oracle's step for step:
//   GDP phase -> (pricing rounds left: scan with the GDP lambda; pairs found ->
//   merge, next phase) -> rule (7) -> finisher if some row is off -> scan with
//   the final lambda (unless that lambda was just scanned) -> none: certified;
//   else merge and continue GDP from lambda (F bits).
extern "C" f2m_status f2m_solve(f2m_ctx* c, f2m_info* info_out) {
  if (!c) return fail(c, F2M_ERR_INVALID_ARG, "NULL context");
  if (cut_count(c))
    return fail(c, F2M_ERR_INVALID_ARG, "the context holds subtour cuts: f2m_solve_subtour drives their solve");
  const auto t0 = std::chrono::steady_clock::now();
  f2m_info info;
  std::memset(&info, 0, sizeof(info));
  const int32_t F = c->p.frac_bits;
  info.frac_bits = F;
  info.batch_shape = -1;
  c->fin_stats = FinisherStats();
  f2m_status status = F2M_OK;
  int64_t last_pairs = 0;  // pairs found by the last scan
  for (;;) {
    int64_t sw = 0;
    f2m_status s = gdp_phase(c, c->p.max_iters, &sw, false, 0, &info.ms_gdp);
    info.iterations += sw;
    info.phases += 1;
    if (s != F2M_OK && s != F2M_ERR_NOT_CONVERGED) { status = s; break; }

    // price the GDP lambda after the first phase and after a phase whose
    // preceding scan found at least n/1024 pairs; otherwise go straight on
    // (the scan with the final lambda finds what is still missing)
    bool clean = false;
    if (c->p.pricing && info.pricing_rounds < c->p.max_pricing_rounds &&
        (info.phases == 1 || last_pairs * 1024 >= c->n)) {
      s = price_internal(c, &info.ms_pricing);
      if (s != F2M_OK) { status = s; break; }
      info.pricing_rounds += 1;
      info.pricing_pairs += c->last_scan_pairs;
      info.certifying_scans += c->last_scan_rows >= 0;
      last_pairs = c->npairs;
      if (c->npairs > 0) {
        const int64_t found = c->npairs;
        s = merge_internal(c, c->d_pairs, c->npairs, &info.ms_merge);
        if (s != F2M_OK) { status = s; break; }
        info.edges_added += found;
        // another GDP phase, unless the first phase's scan found few pairs:
        // the finisher then takes the few new edges from this lambda
        if (info.phases > 1 || found * 1024 >= c->n) continue;
      } else {
        clean = true;
      }
    }

    int64_t bad = 0;
    s = extract_internal(c, &bad, &info.ms_extract);
    if (s != F2M_OK) { status = s; break; }
    if (bad > 0) {
      if (!c->p.finisher) {
        status = F2M_ERR_NOT_CONVERGED;
        fail(c, status, std::to_string(bad) + " nodes violate the degree constraint and the finisher is off");
        break;
      }
      const auto f0 = std::chrono::steady_clock::now();
      int64_t aug = 0;
      s = finisher_internal(c, &aug, nullptr);
      info.ms_finish += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - f0).count();
      info.finisher_calls += 1;
      info.augmentations += aug;
      if (s != F2M_OK) { status = s; break; }
    }
    info.frac_bits = c->fb_cur;
    info.certified = 1;
    if (!c->p.pricing) break;
    if (c->fb_cur == F && clean) { info.certified = 2; break; }
    if (info.pricing_rounds >= c->p.max_pricing_rounds) {
      status = F2M_ERR_NOT_CONVERGED;
      fail(c, status, "pricing rounds exhausted");
      break;
    }
    s = price_internal(c, &info.ms_pricing);
    if (s != F2M_OK) { status = s; break; }
    info.pricing_rounds += 1;
    info.pricing_pairs += c->last_scan_pairs;
    info.certifying_scans += c->last_scan_rows >= 0;
    last_pairs = c->npairs;
    if (c->npairs == 0) { info.certified = 2; break; }
    s = merge_internal(c, c->d_pairs, c->npairs, &info.ms_merge);
    if (s != F2M_OK) { status = s; break; }
    info.edges_added += c->npairs;
    info.certified = 0;
    info.frac_bits = F;
  }
  if (status == F2M_OK || status == F2M_ERR_NOT_CONVERGED) {
    int64_t b2 = 0;
    if (bound_internal(c, &b2) == F2M_OK) info.bound2 = b2;
    info.frac_bits = c->fb_cur;
  }
  info.nnz = c->nnz;
  info.gdp_kernel = c->gdp_kernel;
  info.status = status;
  copy_finisher_stats(c, &info);
  info.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info_out) *info_out = info;
  return status;
}

extern "C" f2m_status f2m_get_lambda(f2m_ctx* c, int32_t* lambda, int32_t* frac_bits) {
  if (!c) return fail(c, F2M_ERR_INVALID_ARG, "NULL context");
  int32_t fb = 0;
  const int32_t* lam = cur_lambda(c, &fb);
  if (frac_bits) *frac_bits = fb;
  if (lambda) {
    CK(c, cudaMemcpyAsync(lambda, lam, sizeof(int32_t) * c->n, cudaMemcpyDefault, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return F2M_OK;
}

extern "C" f2m_status f2m_get_bound(f2m_ctx* c, int64_t* bound2, int32_t* frac_bits) {
  if (!c || !bound2) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  if (frac_bits) *frac_bits = c->fb_cur;
  return bound_internal(c, bound2);
}

extern "C" f2m_status f2m_get_x(f2m_ctx* c, int64_t* nnz_inout, int32_t* row_ptr, int32_t* col,
                                uint8_t* x2, int32_t* cost) {
  if (!c || !nnz_inout) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  const int64_t cap = *nnz_inout;
  *nnz_inout = c->nnz;
  if (!row_ptr && !col && !x2 && !cost) return F2M_OK;
  if ((col || x2 || cost) && cap < c->nnz) return fail(c, F2M_ERR_INVALID_ARG, "capacity below nnz");
  if (row_ptr) CK(c, cudaMemcpyAsync(row_ptr, c->d_rp, sizeof(int32_t) * (c->n + 1), cudaMemcpyDefault, c->st));
  if (x2 && c->nnz) CK(c, cudaMemcpyAsync(x2, c->d_x2, c->nnz, cudaMemcpyDefault, c->st));
  if ((col || cost) && c->nnz) {
    if (c->out_cap < c->nnz) {
      dfree(c->d_out_a);
      dfree(c->d_out_b);
      c->out_cap = c->nnz;
      CK(c, dalloc(&c->d_out_a, c->out_cap));
      CK(c, dalloc(&c->d_out_b, c->out_cap));
    }
    CK(c, launch_split_ec(c->d_ec, c->nnz, c->d_out_a, c->d_out_b, c->st));
    if (col) CK(c, cudaMemcpyAsync(col, c->d_out_a, sizeof(int32_t) * c->nnz, cudaMemcpyDefault, c->st));
    if (cost) CK(c, cudaMemcpyAsync(cost, c->d_out_b, sizeof(int32_t) * c->nnz, cudaMemcpyDefault, c->st));
  }
  CK(c, cudaStreamSynchronize(c->st));
  return F2M_OK;
}
