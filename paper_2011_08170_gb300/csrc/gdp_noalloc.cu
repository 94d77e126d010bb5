// f2m_gdp_noalloc: one GDP phase that allocates no memory.
//
// Some callers cannot call cudaMalloc or cudaFree at the point where they want
// to run GDP: cudaFree waits for the whole device, which a caller driving
// other streams cannot afford; a framework that has reserved the device
// memory for its own pool leaves nothing for cudaMalloc; and a latency-bound
// loop may forbid allocation once it has started.  For them this entry point
// runs the same persistent GDP kernel as f2m_gdp, with its scratch -- the
// second lambda buffer of the Jacobi double buffer and the kernel's control
// block -- in one file-scope device array of fixed size instead of memory
// allocated per context.  The caller passes all inputs and outputs as device
// arrays.  The paper has no counterpart of this; it exists for those callers.
//
// The array is part of the loaded module: every GPU that loads this library
// holds it (kNoAllocScratchInts * 4 bytes, about 1 MiB) until the process exits.
// Host code cannot use the array's name as a device address, so on the first
// call on each device (with that device current) its address is looked up with
// cudaGetSymbolAddress and cached.  All calls share the array and it keeps the
// last call's contents: each call clears the control block before launching,
// and calls that overlap on the GPU race on it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/f2m.h"
#include "f2m_internal.h"

namespace f2m {
namespace {

constexpr int32_t kNoAllocMaxNodes = 1 << 18;  // 262,144 nodes
constexpr int32_t kCtlInts = 64;               // first 256 bytes: the control block
constexpr int64_t kNoAllocScratchInts = kCtlInts + (int64_t)kNoAllocMaxNodes;
static_assert(sizeof(GdpCtl) <= kCtlInts * sizeof(int32_t), "control block must fit its slot");

static __device__ __align__(256) int32_t g_gdp_scratch[kNoAllocScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int32_t* g_scratch_addr[kMaxDevices] = {};  // device address of g_gdp_scratch per device

void set_msg(char* errbuf, int64_t errlen, const char* msg) {
  if (errbuf && errlen > 0) {
    std::strncpy(errbuf, msg, (size_t)errlen - 1);
    errbuf[errlen - 1] = '\0';
  }
}

f2m_status cuda_msg(char* errbuf, int64_t errlen, const char* what, cudaError_t e) {
  if (errbuf && errlen > 0) std::snprintf(errbuf, (size_t)errlen, "%s: %s", what, cudaGetErrorString(e));
  return F2M_ERR_CUDA;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace f2m

using namespace f2m;

extern "C" f2m_status f2m_gdp_noalloc(const int32_t* row_ptr, const int32_t* ec, int32_t n,
                                      int32_t frac_bits, int32_t damping_shift, int64_t max_sweeps,
                                      int32_t* lambda, int64_t* sweeps, int64_t* bound2,
                                      void* stream, char* errbuf, int64_t errlen) {
  set_msg(errbuf, errlen, "");
  if (!row_ptr || !ec || !lambda || !sweeps) {
    set_msg(errbuf, errlen, "NULL argument");
    return F2M_ERR_INVALID_ARG;
  }
  if (n < 4 || n > kNoAllocMaxNodes) {
    if (errbuf && errlen > 0)
      std::snprintf(errbuf, (size_t)errlen,
                    "n = %d is outside [4, %d]: the fixed scratch array of f2m_gdp_noalloc holds "
                    "at most %d nodes; use f2m_create and f2m_gdp for larger graphs",
                    (int)n, (int)kNoAllocMaxNodes, (int)kNoAllocMaxNodes);
    return F2M_ERR_INVALID_ARG;
  }
  if (frac_bits < 1 || frac_bits > 8 || damping_shift < 1 || damping_shift > 8 || max_sweeps < 0) {
    set_msg(errbuf, errlen, "frac_bits and damping_shift must be in 1..8, max_sweeps >= 0");
    return F2M_ERR_INVALID_ARG;
  }
  if (!is_device_pointer(row_ptr) || !is_device_pointer(ec) || !is_device_pointer(lambda)) {
    set_msg(errbuf, errlen, "row_ptr, ec and lambda must be device memory");
    return F2M_ERR_INVALID_ARG;
  }
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) {
    set_msg(errbuf, errlen, "device ordinal beyond the set-up table");
    return F2M_ERR_INVALID_ARG;
  }
  int32_t* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_gdp_scratch);
      if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "cudaGetSymbolAddress", e);
      g_scratch_addr[dev] = static_cast<int32_t*>(p);
    }
    base = g_scratch_addr[dev];
  }
  e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "cudaDeviceGetAttribute", e);

  cudaStream_t st = (cudaStream_t)stream;
  GdpCtl* ctl = reinterpret_cast<GdpCtl*>(base);
  int32_t* lam_other = base + kCtlInts;
  e = cudaMemsetAsync(ctl, 0, sizeof(GdpCtl), st);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "clear control block", e);
  e = launch_gdp(row_ptr, reinterpret_cast<const int2*>(ec), nullptr, 2, lambda, lam_other, n, frac_bits,
                 damping_shift, max_sweeps, ctl, nullptr, nullptr, 0, 4000000000LL, num_sms, st);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "launch", e);
  GdpCtl h;
  e = cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "read control block", e);
  const bool ovf = (h.status & kGdpOverflow) != 0;
  const long long used = ovf ? h.sweeps - 1 : h.sweeps;
  if (used & 1) {  // the last lambda written lives in the scratch half
    e = cudaMemcpyAsync(lambda, lam_other, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "copy lambda back", e);
  }
  *sweeps = h.sweeps;
  if (bound2) *bound2 = h.sweeps > 0 ? h.slot_b2[(h.sweeps - 1) % 3] : 0;
  if (h.status & kGdpTimeout) {
    set_msg(errbuf, errlen, "device-wide barrier wait exceeded its budget");
    return F2M_ERR_TIMEOUT;
  }
  if (ovf) {
    set_msg(errbuf, errlen, "|lambda| reached 2^29");
    return F2M_ERR_OVERFLOW;
  }
  return h.fixed_point ? F2M_OK : F2M_ERR_NOT_CONVERGED;
}
