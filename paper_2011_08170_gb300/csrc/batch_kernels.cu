// Kernels of the batched solver: many instances as one disjoint union of
// segments (contiguous node ranges).  Jacobi sweeps (Eq. 9, Eq. 10) on a
// disjoint union are Jacobi sweeps on each instance, so every instance gets
// exactly the lambda sequence of its own solve; a segment whose sweep changed
// nothing is frozen (its lambda is a fixed point and is left alone) and its
// sweep count is recorded.
//
// gdp_batch_kernel streams the renumbered CSR of every unfrozen segment from
// memory each sweep (the batch does not fit in shared memory): each CTA owns a
// contiguous node range of balanced entry count; G lanes per node read the
// row's 8-byte {col, cost} entries (coalesced) and gather lambda from L2.
#include <climits>

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

// segment of node v: last s with seg_off[s] <= v
__device__ __forceinline__ int segment_of(const int32_t* seg_off, int nseg, int v) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Tiles: contiguous node ranges of one segment with at most kTileEntries
// entries and kTileNodes nodes, dealt round-robin to the CTAs every sweep.
// Per tile the CTA (1) loads every entry with all its threads (many independent
// loads in flight), forms w_e = c_e 2^F - lambda_u and stages it in shared
// memory, then (2) one thread per node takes the top-3 of w_e - lambda_v over
// its row.  Freezing is decided by block 0 after barrier t from the per-segment
// changed counts of sweep t and seen by the other blocks from sweep t+2 on (a
// segment converged at sweep t computes one more sweep, which changes nothing).
template <int T>
__global__ void __launch_bounds__(T)
gdp_batch_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                 const int4* __restrict__ tiles, int32_t ntiles, int32_t nseg, uint8_t* active,
                 unsigned long long* seg_ch, long long* seg_sweeps, int32_t* lam0, int32_t* lam1,
                 int32_t F, int32_t shift, long long max_sweeps, GdpCtl* ctl, long long budget) {
  __shared__ int s_w[kBatchTileEntries];
  __shared__ int s_rp[kBatchTileNodes + 1];
  __shared__ unsigned s_tot[32];
  __shared__ int s_ovf[32];
  __shared__ unsigned s_tile_ch;
  __shared__ int s_stop, s_act;
  const int tid = threadIdx.x, b = blockIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = T / 32;
  const long long div = 1LL << shift;
  volatile GdpCtl* vc = ctl;
  volatile uint8_t* vact = active;

  long long t = 0;
  for (; t < max_sweeps; ++t) {
    const int32_t* lin = (t & 1) ? lam1 : lam0;
    int32_t* lout = (t & 1) ? lam0 : lam1;
    unsigned ch = 0;
    int ovf = 0;
    for (int k = b; k < ntiles; k += gridDim.x) {
      const int4 tl = tiles[k];  // nodes [x, y), segment z, first entry w
      if (tid == 0) { s_act = vact[tl.z]; s_tile_ch = 0; }
      __syncthreads();
      if (!s_act) { __syncthreads(); continue; }
      const int v0 = tl.x, nv = tl.y - tl.x, E0 = tl.w;
      const int ne = __ldg(irp + tl.y) - E0;
      for (int i = tid; i <= nv; i += T) s_rp[i] = __ldg(irp + v0 + i) - E0;
#pragma unroll 4
      for (int e = tid; e < ne; e += T) {
        const int2 q = __ldg(iec + E0 + e);
        s_w[e] = (q.y << F) - ld_cg(lin + q.x);
      }
      __syncthreads();
      for (int i = tid; i < nv; i += T) {
        const int lv = ld_cg(lin + v0 + i);
        int a = INT_MAX, bb = INT_MAX, c = INT_MAX;
        for (int e = s_rp[i]; e < s_rp[i + 1]; ++e) top3_insert_minmax(s_w[e] - lv, a, bb, c);  // Eq. 9
        const long long d = ((long long)bb + (long long)c) / div;  // Eq. 10, truncated toward 0
        const long long nl = (long long)lv + d;
        ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
        lout[v0 + i] = (int32_t)nl;
        if (d != 0) {
          atomicAdd(&s_tile_ch, 1u);
          ++ch;
        }
      }
      __syncthreads();
      if (tid == 0 && s_tile_ch)
        atomicAdd(&seg_ch[(size_t)tl.z * 3 + (t % 3)], (unsigned long long)s_tile_ch);
    }
    ch = warp_sum_u(ch);
    ovf = __any_sync(0xffffffffu, ovf);
    if (lane == 0) { s_tot[warp] = ch; s_ovf[warp] = ovf; }
    __syncthreads();
    if (warp == 0) {
      unsigned y = lane < nwarps ? s_tot[lane] : 0;
      int o = lane < nwarps ? s_ovf[lane] : 0;
      y = warp_sum_u(y);
      o = __any_sync(0xffffffffu, o);
      if (lane == 0) {
        if (y) atomicAdd(&ctl->slot_ch[t % 3], (unsigned long long)y);
        if (o) atomicOr(&ctl->status, kGdpOverflow);
      }
    }
    if (!grid_barrier_counted(&ctl->bar_count, (unsigned)(t + 1) * gridDim.x, budget)) {
      if (tid == 0) atomicOr(&ctl->status, kGdpTimeout);
      break;
    }
    if (b == 0) {  // coordinator: freezes and slot resets for every segment
      for (int s = tid; s < nseg; s += T) {
        volatile unsigned long long* slot = seg_ch + (size_t)s * 3;
        if (vact[s] && slot[t % 3] == 0) {
          vact[s] = 0;
          seg_sweeps[s] = t + 1;
        }
        slot[(t + 2) % 3] = 0;
      }
    }
    if (tid == 0) {
      const unsigned long long chg = vc->slot_ch[t % 3];
      const int st = vc->status;
      if (b == 0) {
        vc->slot_ch[(t + 2) % 3] = 0;
        vc->sweeps = t + 1;
        vc->fixed_point = (chg == 0);
      }
      s_stop = (st != 0) || (chg == 0);
    }
    __syncthreads();
    if (s_stop) break;
  }
}

constexpr int kBatchThreads = 512;

cudaError_t launch_gdp_batch(const int32_t* irp, const int2* iec, const int4* tiles, int32_t ntiles,
                             int32_t B, int32_t nseg, uint8_t* active, unsigned long long* seg_ch,
                             long long* seg_sweeps, int32_t* lam0, int32_t* lam1, int32_t F,
                             int32_t shift, int64_t max_sweeps, GdpCtl* ctl, long long budget,
                             cudaStream_t st) {
  long long ms = max_sweeps;
  void* args[] = {(void*)&irp, (void*)&iec, (void*)&tiles, (void*)&ntiles, (void*)&nseg,
                  (void*)&active, (void*)&seg_ch, (void*)&seg_sweeps, (void*)&lam0, (void*)&lam1,
                  (void*)&F, (void*)&shift, (void*)&ms, (void*)&ctl, (void*)&budget};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)gdp_batch_kernel<kBatchThreads>, dim3(B),
                                              dim3(kBatchThreads), args, 0, st);
  count_launch();
  return e;
}

int batch_blocks_per_sm() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gdp_batch_kernel<kBatchThreads>,
                                                    kBatchThreads, 0) != cudaSuccess)
    return 0;
  return per_sm;
}

// ---- segmented helpers -------------------------------------------------------------

// per-segment bound2 at lam (units 2^-fb); for segments flagged in seg_write
// (NULL = none) also x2 by rule (7) and the count of rows not summing to 4
__global__ void batch_extract_bound_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                           const int32_t* __restrict__ lam, int32_t n, int32_t fb,
                                           const int32_t* __restrict__ seg_off, int32_t nseg,
                                           uint8_t* __restrict__ x2, long long* seg_b2,
                                           unsigned long long* seg_bad,
                                           const uint8_t* __restrict__ seg_write) {
  F2M_GRID_STRIDE(v, n) {
    const int sg = segment_of(seg_off, nseg, (int)v);
    const int write_x = seg_write != nullptr && seg_write[sg];
    const long long lv = lam[v];
    long long acc = 4 * lv;
    int s = 0;
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      const int2 q = ec[e];
      const long long z = ((long long)q.y << fb) - lv - lam[q.x];
      if (z < 0) acc += z;
      const int x = z < 0 ? 2 : (z == 0 ? 1 : 0);
      if (write_x) x2[e] = (uint8_t)x;
      s += x;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&seg_b2[sg]), (unsigned long long)acc);
    if (write_x && s != 4) atomicAdd(&seg_bad[sg], 1ull);
  }
}

cudaError_t launch_batch_extract_bound(const int32_t* rp, const int2* ec, const int32_t* lam,
                                       int32_t n, int32_t fb, const int32_t* seg_off, int32_t nseg,
                                       uint8_t* x2, long long* seg_b2, unsigned long long* seg_bad,
                                       const uint8_t* seg_write, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(seg_b2, 0, sizeof(long long) * nseg, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(seg_bad, 0, sizeof(unsigned long long) * nseg, st);
  if (e != cudaSuccess) return e;
  batch_extract_bound_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp, ec, lam, n, fb, seg_off, nseg, x2,
                                                               seg_b2, seg_bad, seg_write);
  count_launch();
  return cudaGetLastError();
}

// build the union CSR from per-instance local CSRs laid back to back:
//   rp_local: instance s has n_s + 1 offsets starting at seg_off[s] + s
//   col_local: instance s has its entries starting at eoff[s]
__global__ void batch_union_rows_kernel(const int32_t* __restrict__ rp_local,
                                        const int32_t* __restrict__ seg_off,
                                        const int32_t* __restrict__ eoff, int32_t nseg, int32_t n,
                                        int32_t* __restrict__ rp, CheckCtl* ctl) {
  F2M_GRID_STRIDE(v, n + 1) {
    if (v == n) { rp[n] = eoff[nseg]; continue; }
    const int s = segment_of(seg_off, nseg, (int)v);
    const int i = (int)v - seg_off[s];
    const int r = rp_local[seg_off[s] + s + i];
    const int r_end = rp_local[seg_off[s + 1] + s];  // this instance's nnz
    if (r < 0 || r > r_end) { atomicOr(&ctl->flags, 1); atomicMin(&ctl->first_bad, (int)v); }
    rp[v] = eoff[s] + r;
  }
}

__global__ void batch_union_cols_kernel(const int32_t* __restrict__ col_local,
                                        const int32_t* __restrict__ seg_off,
                                        const int32_t* __restrict__ eoff, int32_t nseg,
                                        long long nnz, int32_t* __restrict__ col, CheckCtl* ctl) {
  F2M_GRID_STRIDE(e, nnz) {
    int lo = 0, hi = nseg - 1;  // instance of entry e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (eoff[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int c = col_local[e];
    const int ns = seg_off[lo + 1] - seg_off[lo];
    if (c < 0 || c >= ns) { atomicOr(&ctl->flags, 2); atomicMin(&ctl->first_bad, lo); }
    col[e] = seg_off[lo] + c;
  }
}

cudaError_t launch_batch_union(const int32_t* rp_local, const int32_t* col_local,
                               const int32_t* seg_off, const int32_t* eoff, int32_t nseg, int32_t n,
                               int64_t nnz, int32_t* rp, int32_t* col, CheckCtl* ctl,
                               cudaStream_t st) {
  batch_union_rows_kernel<<<grid_for(n + 1, 256), 256, 0, st>>>(rp_local, seg_off, eoff, nseg, n, rp, ctl);
  count_launch();
  if (nnz > 0) {
    batch_union_cols_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(col_local, seg_off, eoff, nseg, nnz, col, ctl);
    count_launch();
  }
  return cudaGetLastError();
}

// keep the finisher away from excluded segments: zero their surpluses
__global__ void batch_mask_surplus_kernel(int32_t* exl, const int32_t* __restrict__ seg_off,
                                          int32_t nseg, const uint8_t* __restrict__ include,
                                          int32_t n) {
  F2M_GRID_STRIDE(i, n) {
    if (!include[segment_of(seg_off, nseg, (int)i)]) exl[i] = 0;
  }
}

cudaError_t launch_batch_mask_surplus(int32_t* exl, const int32_t* seg_off, int32_t nseg,
                                      const uint8_t* include, int32_t n, cudaStream_t st) {
  batch_mask_surplus_kernel<<<grid_for(n, 256), 256, 0, st>>>(exl, seg_off, nseg, include, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
