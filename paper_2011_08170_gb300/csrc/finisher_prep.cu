// Device-side preparation and scatter for the exact finisher (finisher.cpp).
//
// The finisher walks the candidate graph in the renumbered (Morton) node
// order, where a node's neighbours sit close in memory; rows keep the caller's
// column order, so with ties broken by caller ids its result is the same as on
// the caller's layout.  These kernels build what it needs in one pass each:
//   twin[e]  for e = (i -> j), the entry of (j -> i);
//   y[e]     = 1 if z_e < 0 (arcs of negative reduced cost start saturated);
//   exl[i]   = b_i - #{e in row i : y[e]} (surplus of the left copy of i,
//            b_i = 2 for the fractional 2-matching; the right copy has the
//            opposite value since z is symmetric);
// and map its output back to caller order: x in half units, y[e] + y[twin[e]]
// of the final flow, and lambda at F+1 bits.
#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

#define F2M_GRID_STRIDE(i, count) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (count); \
       i += (long long)gridDim.x * blockDim.x)

static inline int grid_for(long long items, int threads) {
  long long b = (items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

__global__ void fin_twin_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                int32_t n, int32_t* __restrict__ twin, unsigned long long* missing) {
  F2M_GRID_STRIDE(i, n) {
    for (int e = irp[i]; e < irp[i + 1]; ++e) {
      const int j = iec[e].x;
      int f = irp[j];
      const int f1 = irp[j + 1];
      while (f < f1 && iec[f].x != (int)i) ++f;
      twin[e] = f < f1 ? f : -1;
      if (f >= f1) atomicAdd(missing, 1ull);
    }
  }
}

__global__ void fin_init_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                const int32_t* __restrict__ lam, const int32_t* __restrict__ bdeg,
                                const int32_t* __restrict__ perm, int32_t n, int32_t F,
                                uint8_t* __restrict__ y, int32_t* __restrict__ exl) {
  F2M_GRID_STRIDE(i, n) {
    const long long li = lam[i];
    int cnt = 0;
    for (int e = irp[i]; e < irp[i + 1]; ++e) {
      const int2 q = iec[e];
      const long long z = ((long long)q.y << F) - li - lam[q.x];
      y[e] = (uint8_t)(z < 0);
      cnt += (z < 0);
    }
    exl[i] = (bdeg ? bdeg[perm[i]] : 2) - cnt;
  }
}

__global__ void fin_scatter_x_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ irp,
                                     const int32_t* __restrict__ perm, int32_t n,
                                     const uint8_t* __restrict__ y, const int32_t* __restrict__ twin,
                                     uint8_t* __restrict__ x_out,
                                     const int32_t* __restrict__ seg_off, int32_t nseg,
                                     const uint8_t* __restrict__ include) {
  F2M_GRID_STRIDE(i, n) {
    if (include) {  // segments the finisher left alone keep their x
      int lo = 0, hi = nseg - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= (int)i) lo = mid; else hi = mid - 1;
      }
      if (!include[lo]) continue;
    }
    const int dst = rp[perm[i]], src = irp[i], cnt = irp[i + 1] - src;
    for (int k = 0; k < cnt; ++k) x_out[dst + k] = (uint8_t)(y[src + k] + y[twin[src + k]]);
  }
}

cudaError_t fin_build_twin(const GdpPlan& p, int32_t* twin, unsigned long long* missing, cudaStream_t st) {
  fin_twin_kernel<<<grid_for(p.n, 128), 128, 0, st>>>(p.irp, p.iec, p.n, twin, missing);
  count_launch();
  return cudaGetLastError();
}

cudaError_t fin_prepare(const GdpPlan& p, const int32_t* lam_caller, const int32_t* bdeg_caller,
                        int32_t F, int32_t* lam_int, uint8_t* y, int32_t* exl, cudaStream_t st) {
  gather_perm(lam_caller, p.perm, p.n, lam_int, st);
  fin_init_kernel<<<grid_for(p.n, 128), 128, 0, st>>>(p.irp, p.iec, lam_int, bdeg_caller, p.perm,
                                                      p.n, F, y, exl);
  count_launch();
  return cudaGetLastError();
}

cudaError_t fin_scatter(const GdpPlan& p, const int32_t* rp, const uint8_t* y_int,
                        const int32_t* twin, const int32_t* lam2_int, uint8_t* x_out,
                        int32_t* lam2_out, const int32_t* seg_off, int32_t nseg,
                        const uint8_t* include, cudaStream_t st) {
  fin_scatter_x_kernel<<<grid_for(p.n, 128), 128, 0, st>>>(rp, p.irp, p.perm, p.n, y_int, twin, x_out,
                                                           seg_off, nseg, include);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return scatter_perm(lam2_int, p.perm, p.n, lam2_out, st);
}

}  // namespace f2m
