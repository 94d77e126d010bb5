// C ABI of the candidate-graph builder (k nearest neighbours, Section 5.3) and
// of the learned warm start (features, network, training, lambda0).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/f2m.h"
#include "ctx_internal.h"
#include "f2m_internal.h"

using namespace f2m;

struct f2m_mlp {
  cudaStream_t st = nullptr;
  int num_sms = 0;
  float* master = nullptr;   // fp32 parameters
  float* m1 = nullptr;       // Adam moments
  float* m2 = nullptr;
  uint8_t* img = nullptr;    // bf16 operand images of W1, W2, W2^T
  float* partial = nullptr;  // per-CTA partial gradients [num_sms][kMlpParams + 1]
  float* grad = nullptr;     // [kMlpParams + 1]
  long long* step = nullptr; // Adam steps taken
  int* status = nullptr;     // bit 0: a tensor-core wait gave up
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A caller array seen from the device: the pointer itself if it is device
// memory, else a stream-ordered staging copy (copied in on request, copied back
// by flush()).
template <typename T>
struct DevView {
  T* user = nullptr;
  T* d = nullptr;
  size_t count = 0;
  bool staged = false;
  cudaStream_t st = nullptr;
  cudaError_t open(T* p, size_t cnt, bool copy_in, cudaStream_t s) {
    user = p;
    count = cnt;
    st = s;
    if (is_device_ptr(p)) {
      d = p;
      return cudaSuccess;
    }
    staged = true;
    cudaError_t e = cudaMallocAsync((void**)&d, sizeof(T) * (cnt ? cnt : 1), s);
    if (e == cudaSuccess && copy_in && cnt)
      e = cudaMemcpyAsync(d, p, sizeof(T) * cnt, cudaMemcpyHostToDevice, s);
    return e;
  }
  cudaError_t flush() {
    if (!staged || !count) return cudaSuccess;
    return cudaMemcpyAsync(user, d, sizeof(T) * count, cudaMemcpyDeviceToHost, st);
  }
  ~DevView() {
    if (staged && d) cudaFreeAsync(d, st);
  }
};

f2m_status mlp_fail(f2m_mlp* m, f2m_status s, const std::string& msg) {
  if (m) m->err = msg;
  return fail(nullptr, s, msg);
}

f2m_status mlp_cuda(f2m_mlp* m, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return mlp_fail(m, e == cudaErrorMemoryAllocation ? F2M_ERR_OOM : F2M_ERR_CUDA, msg);
}

#define MCK(m, call)                                         \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return mlp_cuda((m), e_, #call);  \
  } while (0)

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

f2m_status check_status(f2m_mlp* m) {
  int h = 0;
  MCK(m, cudaMemcpyAsync(&h, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  MCK(m, cudaStreamSynchronize(m->st));
  if (h) return mlp_fail(m, F2M_ERR_TIMEOUT, "a tensor-core completion wait gave up");
  return F2M_OK;
}

}  // namespace

// ---- k nearest neighbours ----------------------------------------------------------

extern "C" f2m_status f2m_knn(const int32_t* xy, int32_t n, int32_t k, int32_t* nbr, int64_t* d2,
                              void* stream) {
  if (!xy || !nbr) return fail(nullptr, F2M_ERR_INVALID_ARG, "NULL argument");
  if (k < 1 || k > kKnnMax) return fail(nullptr, F2M_ERR_INVALID_ARG, "k must be in 1..32");
  if (n <= k || n >= (1 << 24)) return fail(nullptr, F2M_ERR_INVALID_ARG, "n must be in (k, 2^24)");
  cudaStream_t st = (cudaStream_t)stream;
  DevView<int2> vxy;
  DevView<int32_t> vn;
  DevView<int64_t> vd;
  cudaError_t e = vxy.open((int2*)xy, n, true, st);
  if (e == cudaSuccess) e = vn.open(nbr, (size_t)n * k, false, st);
  if (e == cudaSuccess && d2) e = vd.open(d2, (size_t)n * k, false, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_knn: buffers");
  // coordinates must be inside the grid
  CheckCtl* ctl = nullptr;
  e = cudaMallocAsync((void**)&ctl, sizeof(CheckCtl), st);
  CheckCtl h{0, 0x7fffffff};
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, &h, sizeof h, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_check_points(vxy.d, n, ctl, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(ctl, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_knn: check");
  if (h.flags) return fail(nullptr, F2M_ERR_INVALID_ARG, "coordinate outside [0, 2^20) at node " + std::to_string(h.first_bad));
  e = knn_device(vxy.d, n, k, vn.d, d2 ? (long long*)vd.d : nullptr, st);
  if (e == cudaSuccess) e = vn.flush();
  if (e == cudaSuccess && d2) e = vd.flush();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_knn");
  return F2M_OK;
}

extern "C" f2m_status f2m_knn_csr(const int32_t* xy, int32_t n, int32_t k, int32_t* row_ptr,
                                  int32_t* col, int64_t* nnz, void* stream) {
  if (!xy || !row_ptr || !col || !nnz) return fail(nullptr, F2M_ERR_INVALID_ARG, "NULL argument");
  if (k < 1 || k > kKnnMax) return fail(nullptr, F2M_ERR_INVALID_ARG, "k must be in 1..32");
  if (n <= k || 2LL * n * k >= (1LL << 31)) return fail(nullptr, F2M_ERR_INVALID_ARG, "n must be > k and 2nk < 2^31");
  cudaStream_t st = (cudaStream_t)stream;
  DevView<int2> vxy;
  DevView<int32_t> vrp, vcol;
  cudaError_t e = vxy.open((int2*)xy, n, true, st);
  if (e == cudaSuccess) e = vrp.open(row_ptr, (size_t)n + 1, false, st);
  if (e == cudaSuccess) e = vcol.open(col, 2 * (size_t)n * k, false, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_knn_csr: buffers");
  CheckCtl* ctl = nullptr;
  e = cudaMallocAsync((void**)&ctl, sizeof(CheckCtl), st);
  CheckCtl h{0, 0x7fffffff};
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, &h, sizeof h, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_check_points(vxy.d, n, ctl, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(ctl, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_knn_csr: check");
  if (h.flags) return fail(nullptr, F2M_ERR_INVALID_ARG, "coordinate outside [0, 2^20) at node " + std::to_string(h.first_bad));
  int64_t m = 0;
  e = knn_csr_device(vxy.d, n, k, vrp.d, vcol.d, &m, st);
  if (e == cudaSuccess) {
    vcol.count = (size_t)m;
    e = vrp.flush();
  }
  if (e == cudaSuccess) e = vcol.flush();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_knn_csr");
  *nnz = m;
  return F2M_OK;
}

extern "C" f2m_status f2m_features(const int32_t* xy, int32_t n, float* feat, float* scale, void* stream) {
  if (!xy || !feat || !scale) return fail(nullptr, F2M_ERR_INVALID_ARG, "NULL argument");
  if (n <= kFeatures || n >= (1 << 24)) return fail(nullptr, F2M_ERR_INVALID_ARG, "n must be in (16, 2^24)");
  cudaStream_t st = (cudaStream_t)stream;
  DevView<int2> vxy;
  DevView<float> vf, vs;
  cudaError_t e = vxy.open((int2*)xy, n, true, st);
  if (e == cudaSuccess) e = vf.open(feat, (size_t)n * kFeatures, false, st);
  if (e == cudaSuccess) e = vs.open(scale, (size_t)n, false, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_features: buffers");
  CheckCtl* ctl = nullptr;
  e = cudaMallocAsync((void**)&ctl, sizeof(CheckCtl), st);
  CheckCtl h{0, 0x7fffffff};
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, &h, sizeof h, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_check_points(vxy.d, n, ctl, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(ctl, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_features: check");
  if (h.flags) return fail(nullptr, F2M_ERR_INVALID_ARG, "coordinate outside [0, 2^20) at node " + std::to_string(h.first_bad));
  e = features_device(vxy.d, n, vf.d, vs.d, st);
  if (e == cudaSuccess) e = vf.flush();
  if (e == cudaSuccess) e = vs.flush();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "f2m_features");
  return F2M_OK;
}

// ---- the network ------------------------------------------------------------------

extern "C" void f2m_mlp_destroy(f2m_mlp* m) {
  if (!m) return;
  DevSyncedScope synced;  // one wait for the device, then every block goes to the cache
  dfree(m->master); dfree(m->m1); dfree(m->m2); dfree(m->img); dfree(m->partial);
  dfree(m->grad); dfree(m->step); dfree(m->status);
  if (m->ev0) cudaEventDestroy(m->ev0);
  if (m->ev1) cudaEventDestroy(m->ev1);
  delete m;
}

extern "C" const char* f2m_mlp_last_error(const f2m_mlp* m) { return m ? m->err.c_str() : ""; }

extern "C" f2m_status f2m_mlp_create(const float* params, void* stream, f2m_mlp** out) {
  if (!out) return fail(nullptr, F2M_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!params) return fail(nullptr, F2M_ERR_INVALID_ARG, "params is NULL");
  f2m_mlp* m = new (std::nothrow) f2m_mlp();
  if (!m) return fail(nullptr, F2M_ERR_OOM, "host allocation");
  m->st = (cudaStream_t)stream;
  m->num_sms = device_sms();
  std::vector<float> h(kMlpParams);
  cudaError_t e = cudaMemcpyAsync(h.data(), params, sizeof(float) * kMlpParams, cudaMemcpyDefault, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e == cudaSuccess) e = dalloc(&m->master, kMlpParams);
  if (e == cudaSuccess) e = dalloc(&m->m1, kMlpParams);
  if (e == cudaSuccess) e = dalloc(&m->m2, kMlpParams);
  if (e == cudaSuccess) e = dalloc(&m->img, kMlpImgBytes);
  if (e == cudaSuccess) e = dalloc(&m->partial, (int64_t)(m->num_sms > 0 ? m->num_sms : 1) * (kMlpParams + 1));
  if (e == cudaSuccess) e = dalloc(&m->grad, kMlpParams + 1);
  if (e == cudaSuccess) e = dalloc(&m->step, 1);
  if (e == cudaSuccess) e = dalloc(&m->status, 1);
  if (e == cudaSuccess) e = cudaEventCreate(&m->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&m->ev1);
  if (e != cudaSuccess) {
    f2m_status s = mlp_cuda(nullptr, e, "f2m_mlp_create");
    f2m_mlp_destroy(m);
    return s;
  }
  for (int i = 0; i < kMlpParams; ++i) {
    if (!std::isfinite(h[i])) {
      f2m_mlp_destroy(m);
      return fail(nullptr, F2M_ERR_INVALID_ARG, "parameter " + std::to_string(i) + " is not finite");
    }
  }
  e = cudaMemcpyAsync(m->master, h.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, sizeof(float) * kMlpParams, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, sizeof(float) * kMlpParams, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->img, 0, kMlpImgBytes, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->step, 0, sizeof(long long), m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(int), m->st);
  if (e == cudaSuccess) e = mlp_pack(m->master, m->img, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) {
    f2m_status s = mlp_cuda(nullptr, e, "f2m_mlp_create: upload");
    f2m_mlp_destroy(m);
    return s;
  }
  *out = m;
  return F2M_OK;
}

extern "C" f2m_status f2m_mlp_get_params(f2m_mlp* m, float* out) {
  if (!m || !out) return mlp_fail(m, F2M_ERR_INVALID_ARG, "NULL argument");
  MCK(m, cudaMemcpyAsync(out, m->master, sizeof(float) * kMlpParams, cudaMemcpyDefault, m->st));
  MCK(m, cudaStreamSynchronize(m->st));
  return F2M_OK;
}

extern "C" f2m_status f2m_mlp_forward(f2m_mlp* m, const float* feat, int64_t count, float* y) {
  if (!m || !feat || !y) return mlp_fail(m, F2M_ERR_INVALID_ARG, "NULL argument");
  if (count < 0) return mlp_fail(m, F2M_ERR_INVALID_ARG, "count < 0");
  if (count == 0) return F2M_OK;
  DevView<float> vf, vy;
  MCK(m, vf.open((float*)feat, (size_t)count * kFeatures, true, m->st));
  MCK(m, vy.open(y, (size_t)count, false, m->st));
  MCK(m, mlp_forward(m->img, m->master, vf.d, count, vy.d, nullptr, nullptr, 0, m->num_sms, m->status, m->st));
  MCK(m, vy.flush());
  return check_status(m);
}

extern "C" f2m_status f2m_mlp_grad(f2m_mlp* m, const float* feat, const float* target, int64_t count,
                                   float* grad, float* loss) {
  if (!m || !feat || !target || !grad) return mlp_fail(m, F2M_ERR_INVALID_ARG, "NULL argument");
  if (count < 1 || count >= (1LL << 31)) return mlp_fail(m, F2M_ERR_INVALID_ARG, "count must be in [1, 2^31)");
  DevView<float> vf, vt, vg, vl;
  MCK(m, vf.open((float*)feat, (size_t)count * kFeatures, true, m->st));
  MCK(m, vt.open((float*)target, (size_t)count, true, m->st));
  MCK(m, vg.open(grad, kMlpParams, false, m->st));
  const int grid = mlp_grid(m->num_sms, count);
  MCK(m, mlp_train_launch(m->img, m->master, vf.d, vt.d, nullptr, 0, count, 2.f / (float)count,
                          m->partial, grid, nullptr, m->status, m->st));
  MlpAdam hp{};
  MCK(m, mlp_reduce_launch(m->partial, grid, vg.d, m->master, m->m1, m->m2, m->img, nullptr, hp,
                           m->grad + kMlpParams, m->st));
  MCK(m, vg.flush());
  if (loss) {
    float ls = 0.f;
    MCK(m, cudaMemcpyAsync(&ls, m->grad + kMlpParams, sizeof(float), cudaMemcpyDeviceToHost, m->st));
    MCK(m, cudaStreamSynchronize(m->st));
    const float mean = ls / (float)count;
    MCK(m, cudaMemcpyAsync(loss, &mean, sizeof(float), cudaMemcpyDefault, m->st));
  }
  return check_status(m);
}

extern "C" f2m_status f2m_mlp_train(f2m_mlp* m, const float* feat, const float* target, int64_t count,
                                    const f2m_train_params* tp, float* epoch_loss) {
  if (!m || !feat || !target || !tp) return mlp_fail(m, F2M_ERR_INVALID_ARG, "NULL argument");
  if (count < 1 || count >= (1LL << 31)) return mlp_fail(m, F2M_ERR_INVALID_ARG, "count must be in [1, 2^31)");
  if (tp->epochs < 0 || tp->batch < 128 || !(tp->lr > 0.f) || !(tp->beta1 >= 0.f && tp->beta1 < 1.f) ||
      !(tp->beta2 >= 0.f && tp->beta2 < 1.f) || !(tp->eps > 0.f) || !(tp->lr_final_frac >= 0.f))
    return mlp_fail(m, F2M_ERR_INVALID_ARG, "bad training parameters");
  DevView<float> vf, vt;
  MCK(m, vf.open((float*)feat, (size_t)count * kFeatures, true, m->st));
  MCK(m, vt.open((float*)target, (size_t)count, true, m->st));
  const long long batch = tp->batch;
  const long long steps = (count + batch - 1) / batch;
  const int grid = mlp_grid(m->num_sms, batch);
  uint64_t *keys = nullptr, *skeys = nullptr;
  int32_t *idx = nullptr, *perm = nullptr;
  float* loss_log = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  MCK(m, sort_pairs_u64(nullptr, tmp_bytes, nullptr, nullptr, nullptr, nullptr, (int32_t)count, 64, m->st));
  MCK(m, cudaMallocAsync((void**)&keys, sizeof(uint64_t) * count, m->st));
  MCK(m, cudaMallocAsync((void**)&skeys, sizeof(uint64_t) * count, m->st));
  MCK(m, cudaMallocAsync((void**)&idx, sizeof(int32_t) * count, m->st));
  MCK(m, cudaMallocAsync((void**)&perm, sizeof(int32_t) * count, m->st));
  MCK(m, cudaMallocAsync((void**)&loss_log, sizeof(float) * (steps * (tp->epochs > 0 ? tp->epochs : 1)), m->st));
  MCK(m, cudaMallocAsync(&tmp, tmp_bytes ? tmp_bytes : 1, m->st));
  long long t0 = 0;
  MCK(m, cudaMemcpyAsync(&t0, m->step, sizeof(long long), cudaMemcpyDeviceToHost, m->st));
  MCK(m, cudaStreamSynchronize(m->st));
  MlpAdam hp{tp->lr, tp->beta1, tp->beta2, tp->eps, tp->lr_final_frac, t0 + steps * tp->epochs, t0};
  f2m_status s = F2M_OK;
  for (int ep = 0; ep < tp->epochs && s == F2M_OK; ++ep) {
    cudaError_t e = mlp_perm_keys(tp->seed * 0x100000001B3ull + (uint64_t)ep * 0x9E3779B97F4A7C15ull, count,
                                  keys, idx, m->st);
    size_t b = tmp_bytes;
    if (e == cudaSuccess) e = sort_pairs_u64(tmp, b, keys, skeys, idx, perm, (int32_t)count, 64, m->st);
    for (long long k = 0; k < steps && e == cudaSuccess; ++k) {
      const long long s0 = k * batch;
      const long long cnt = count - s0 < batch ? count - s0 : batch;
      e = mlp_train_launch(m->img, m->master, vf.d, vt.d, perm, s0, cnt, 2.f / (float)cnt, m->partial, grid,
                           m->step, m->status, m->st);
      if (e == cudaSuccess)
        e = mlp_reduce_launch(m->partial, grid, nullptr, m->master, m->m1, m->m2, m->img, m->step, hp,
                              loss_log, m->st);
    }
    if (e != cudaSuccess) s = mlp_cuda(m, e, "f2m_mlp_train");
    if (s == F2M_OK) s = check_status(m);
    if (s == F2M_OK && epoch_loss) {
      std::vector<float> h(steps);
      e = cudaMemcpyAsync(h.data(), loss_log + ep * steps, sizeof(float) * steps, cudaMemcpyDeviceToHost, m->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
      if (e != cudaSuccess) s = mlp_cuda(m, e, "f2m_mlp_train: loss");
      double acc = 0.0;
      for (float v : h) acc += v;
      epoch_loss[ep] = (float)(acc / (double)count);
    }
  }
  cudaFreeAsync(keys, m->st);
  cudaFreeAsync(skeys, m->st);
  cudaFreeAsync(idx, m->st);
  cudaFreeAsync(perm, m->st);
  cudaFreeAsync(loss_log, m->st);
  cudaFreeAsync(tmp, m->st);
  cudaStreamSynchronize(m->st);
  return s;
}

// ---- warm start of a context --------------------------------------------------------

extern "C" f2m_status f2m_warm_start(f2m_ctx* c, f2m_mlp* m, double* ms) {
  if (!c || !m) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  if (c->n <= kFeatures) return fail(c, F2M_ERR_INVALID_ARG, "warm start needs n > 16");
  // the network's last update (on its own stream) comes first
  CK(c, cudaEventRecord(m->ev0, m->st));
  CK(c, cudaStreamWaitEvent(c->st, m->ev0, 0));
  float* feat = nullptr;
  float* scale = nullptr;
  CK(c, cudaEventRecord(c->ev0, c->st));
  c->lam_version += 1;
  CK(c, cudaMallocAsync((void**)&feat, sizeof(float) * (size_t)c->n * kFeatures, c->st));
  CK(c, cudaMallocAsync((void**)&scale, sizeof(float) * (size_t)c->n, c->st));
  cudaError_t e = features_device(c->d_xy, c->n, feat, scale, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(int), c->st);
  if (e == cudaSuccess)
    e = mlp_forward(m->img, m->master, feat, c->n, nullptr, scale, c->d_lam[c->cur], c->p.frac_bits,
                    c->num_sms, m->status, c->st);
  cudaFreeAsync(feat, c->st);
  cudaFreeAsync(scale, c->st);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev1, c->st);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, m->status, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "f2m_warm_start");
  if (h) return fail(c, F2M_ERR_TIMEOUT, "a tensor-core completion wait gave up");
  c->fb_cur = c->p.frac_bits;
  if (ms) {
    float t = 0.f;
    cudaEventElapsedTime(&t, c->ev0, c->ev1);
    *ms = t;
  }
  return F2M_OK;
}
