// f2m_gdp_noalloc: one GDP phase that allocates no memory.
//
// Some callers cannot call cudaMalloc or cudaFree at the point where they want
// to run GDP: cudaFree waits for the whole device, which a caller driving
// other streams cannot afford; a framework that has reserved the device
// memory for its own pool leaves nothing for cudaMalloc; and a latency-bound
// loop may forbid allocation once it has started.  For them this entry point
// runs the same persistent GDP kernel as f2m_gdp, with its scratch -- the
// second lambda buffer of the Jacobi double buffer, the kernel's control
// block and the flags of the input check -- in one file-scope device array of
// fixed size instead of memory allocated per context.  The caller passes all
// inputs and outputs as device arrays.  The paper has no counterpart of this;
// it exists for those callers.
//
// The array is part of the loaded module: every GPU that loads this library
// holds it (kNoAllocScratchInts * 4 bytes, about 1 MiB) until the process exits.
// Host code cannot use the array's name as a device address, so every call
// looks the address up with cudaGetSymbolAddress on the current device (a
// cheap table lookup once the module is loaded; it stays right across a
// device reset, which reloads the module).  All calls share the array and it
// keeps the last call's contents: each call clears the control slot before
// launching, and calls that overlap on the GPU race on it.
//
// Before the GDP kernel runs, a check kernel validates the caller's arrays
// (every read inside [0, n] of row_ptr and [0, nnz) of ec): row offsets from 0
// to nnz and nondecreasing, columns in [0, n) and not the row itself, degree
// at least 3 (Eq. 10 needs a third value), costs in [0, 2^(29-F)) and
// |lambda| < 2^29, so that z = c 2^F - lambda_u - lambda_v (Eq. 9) fits int32.
// A violation returns INVALID_ARG and the GDP kernel is not launched.
#include <climits>
#include <cstdio>
#include <cstring>

#include "../../include/f2m.h"
#include "f2m_internal.h"

namespace f2m {
namespace {

constexpr int32_t kNoAllocMaxNodes = 1 << 18;  // 262,144 nodes
constexpr int32_t kCtlInts = 64;               // first 256 bytes: the control slot
constexpr int32_t kCheckInt = 56;              // CheckCtl in the slot's last 32 bytes
constexpr int64_t kNoAllocScratchInts = kCtlInts + (int64_t)kNoAllocMaxNodes;
static_assert(sizeof(GdpCtl) <= kCheckInt * sizeof(int32_t), "control block must fit before the check flags");
static_assert(sizeof(CheckCtl) <= (kCtlInts - kCheckInt) * sizeof(int32_t), "check flags must fit the slot");

static __device__ __align__(256) int32_t g_gdp_scratch[kNoAllocScratchInts];

enum NoAllocBits { kBadCost = 1 << 12, kBadLambda = 1 << 13 };

// One thread per node v: its row offsets, and only if they lie inside
// [0, nnz], its entries and its lambda.  Reads stay in bounds whatever the
// contents of row_ptr.
__global__ void noalloc_check_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                     int64_t nnz, int32_t n, const int32_t* __restrict__ lam,
                                     int32_t cost_limit, CheckCtl* chk) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int flags = 0;
  const long long b = rp[v], e = rp[v + 1];
  if ((v == 0 && b != 0) || (v == n - 1 && e != nnz) || b < 0 || b > e || e > nnz) {
    flags |= kBadRowPtr;
  } else {
    if (e - b < 3) flags |= kLowDegree;
    for (long long q = b; q < e; ++q) {
      const int2 x = ec[q];
      if (x.x < 0 || x.x >= n) flags |= kBadCol;
      else if (x.x == v) flags |= kSelfLoop;
      if (x.y < 0 || x.y >= cost_limit) flags |= kBadCost;
    }
  }
  const long long l = lam[v];
  if (l >= kLamLimit || l <= -kLamLimit) flags |= kBadLambda;
  if (flags) {
    atomicOr(&chk->flags, flags);
    atomicMin(&chk->first_bad, v);
  }
}

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

extern "C" f2m_status f2m_gdp_noalloc(const int32_t* row_ptr, const int32_t* ec, int64_t nnz, int32_t n,
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
  if (nnz < 3LL * n || nnz > INT32_MAX) {
    set_msg(errbuf, errlen, "nnz must be in [3 n, 2^31 - 1] (every row needs at least 3 entries)");
    return F2M_ERR_INVALID_ARG;
  }
  if (!is_device_pointer(row_ptr) || !is_device_pointer(ec) || !is_device_pointer(lambda)) {
    set_msg(errbuf, errlen, "row_ptr, ec and lambda must be device memory");
    return F2M_ERR_INVALID_ARG;
  }
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "cudaGetDevice", e);
  void* sym = nullptr;
  e = cudaGetSymbolAddress(&sym, g_gdp_scratch);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "cudaGetSymbolAddress", e);
  int32_t* base = static_cast<int32_t*>(sym);
  e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "cudaDeviceGetAttribute", e);

  cudaStream_t st = (cudaStream_t)stream;
  GdpCtl* ctl = reinterpret_cast<GdpCtl*>(base);
  CheckCtl* chk = reinterpret_cast<CheckCtl*>(base + kCheckInt);
  int32_t* lam_other = base + kCtlInts;
  e = cudaMemsetAsync(base, 0, kCtlInts * sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&chk->first_bad, 0x7f, sizeof(int), st);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "clear control slot", e);
  noalloc_check_kernel<<<(n + 255) / 256, 256, 0, st>>>(row_ptr, reinterpret_cast<const int2*>(ec), nnz, n,
                                                        lambda, 1 << (29 - frac_bits), chk);
  count_launch();
  CheckCtl hc{};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, chk, sizeof(hc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_msg(errbuf, errlen, "input check", e);
  if (hc.flags) {
    const char* what = (hc.flags & kBadRowPtr)  ? "row_ptr not nondecreasing from 0 to nnz"
                       : (hc.flags & kBadCol)    ? "column outside [0, n)"
                       : (hc.flags & kSelfLoop)  ? "self-loop"
                       : (hc.flags & kLowDegree) ? "degree below 3"
                       : (hc.flags & kBadCost)   ? "cost outside [0, 2^(29 - frac_bits))"
                                                 : "|lambda| >= 2^29";
    if (errbuf && errlen > 0)
      std::snprintf(errbuf, (size_t)errlen, "invalid input at node %d: %s", hc.first_bad, what);
    return F2M_ERR_INVALID_ARG;
  }
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
