// Candidate-graph kernels: input validation, the cost table, and the union of
// the CSR with the pairs found by pricing (rows kept sorted and unique, so the
// result does not depend on the order in which pairs were appended).
#include <climits>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

static inline int grid_for(long long items, int threads) {
  long long b = (items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

#define F2M_GRID_STRIDE(i, count) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (count); \
       i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ void flag(CheckCtl* ctl, int bit, long long where) {
  atomicOr(&ctl->flags, bit);
  atomicMin(&ctl->first_bad, (int)(where < INT_MAX ? where : INT_MAX));
}

// pass 1: row offsets monotone and in [0, nnz], coordinates in range
__global__ void check_rowptr_kernel(const int2* xy, const int32_t* rp, int32_t n, int64_t nnz,
                                    CheckCtl* ctl) {
  F2M_GRID_STRIDE(v, n) {
    const int a = rp[v], b = rp[v + 1];
    if (a < 0 || b < a || (long long)b > nnz || (v == 0 && a != 0) || (v == n - 1 && b != nnz))
      flag(ctl, kBadRowPtr, v);
    const int2 p = xy[v];
    if (p.x < 0 || p.y < 0 || p.x >= kCoordLimit || p.y >= kCoordLimit) flag(ctl, kBadCoord, v);
  }
}

// coordinates only (for calls that take points without a graph)
__global__ void check_points_kernel(const int2* xy, int32_t n, CheckCtl* ctl) {
  F2M_GRID_STRIDE(v, n) {
    const int2 p = xy[v];
    if (p.x < 0 || p.y < 0 || p.x >= kCoordLimit || p.y >= kCoordLimit) flag(ctl, kBadCoord, v);
  }
}

// pass 2 (row offsets valid): columns, order, self-loops, degree, symmetry
__global__ void check_rows_kernel(const int32_t* rp, const int32_t* col, int32_t n, CheckCtl* ctl) {
  F2M_GRID_STRIDE(v, n) {
    const int a = rp[v], b = rp[v + 1];
    if (b - a < 3) flag(ctl, kLowDegree, v);
    int prev = -1;
    for (int e = a; e < b; ++e) {
      const int c = col[e];
      if (c < 0 || c >= n) { flag(ctl, kBadCol, v); continue; }
      if (c == v) flag(ctl, kSelfLoop, v);
      if (c <= prev) flag(ctl, kUnsorted, v);
      prev = c;
      // reverse entry (c -> v) must exist; row c is searched only if sorted
      int lo = rp[c], hi = rp[c + 1] - 1, found = 0;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int cm = col[mid];
        if (cm == v) { found = 1; break; }
        if (cm < v) lo = mid + 1; else hi = mid - 1;
      }
      if (!found) {
        // unsorted rows make binary search unreliable; fall back to a scan
        for (int f = rp[c]; f < rp[c + 1] && !found; ++f) found = (col[f] == v);
        if (!found) flag(ctl, kAsymmetric, v);
      }
    }
  }
}

cudaError_t launch_check_points(const int2* xy, int32_t n, CheckCtl* ctl, cudaStream_t st) {
  check_points_kernel<<<grid_for(n, 256), 256, 0, st>>>(xy, n, ctl);
  count_launch();
  return cudaGetLastError();
}

// degree requirements: 1 <= b_v and b_v + 1 <= deg(v) (the (b_v+1)-th value of
// the row must exist, Section 3)
__global__ void check_degrees_kernel(const int32_t* rp, const int32_t* bdeg, int32_t n, CheckCtl* ctl,
                                     unsigned long long* bmax) {
  F2M_GRID_STRIDE(v, n) {
    const int bv = bdeg[v];
    if (bv < 1 || (long long)bv + 1 > (long long)rp[v + 1] - rp[v]) flag(ctl, kBadDegreeReq, v);
    else atomicMax(bmax, (unsigned long long)bv);
  }
}

cudaError_t launch_check_degrees(const int32_t* rp, const int32_t* bdeg, int32_t n, CheckCtl* ctl,
                                 unsigned long long* bmax, cudaStream_t st) {
  check_degrees_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp, bdeg, n, ctl, bmax);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_check(const int2* xy, const int32_t* rp, const int32_t* col, int32_t n,
                         int64_t nnz, CheckCtl* ctl, cudaStream_t st) {
  // two passes; the host reads ctl between them (pass 2 trusts the row offsets)
  if (col == nullptr) {
    check_rowptr_kernel<<<grid_for(n, 256), 256, 0, st>>>(xy, rp, n, nnz, ctl);
    count_launch();
  } else {
    check_rows_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp, col, n, ctl);
    count_launch();
  }
  return cudaGetLastError();
}

// ec[e] = {col[e], c(v, col[e])}, one thread per entry with the row found by
// a binary search of rp (entries of one warp share rows, so it stays cached)
__global__ void build_ec_kernel(const int2* __restrict__ xy, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, int32_t n, long long nnz,
                                int2* __restrict__ ec) {
  F2M_GRID_STRIDE(e, nnz) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rp[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int c = col[e];
    ec[e] = make_int2(c, exact_cost(xy[lo], xy[c]));
  }
}

cudaError_t launch_build_ec(const int2* xy, const int32_t* rp, const int32_t* col, int32_t n,
                            int2* ec, cudaStream_t st) {
  int32_t nnz_host = 0;
  cudaError_t err = cudaMemcpyAsync(&nnz_host, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return err;
  if (nnz_host == 0) return cudaSuccess;
  build_ec_kernel<<<grid_for(nnz_host, 256), 256, 0, st>>>(xy, rp, col, n, nnz_host, ec);
  count_launch();
  return cudaGetLastError();
}

// ---- exclusive scan of int32 (m+1 outputs, out[m] = total) -------------------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

size_t scan_scratch_ints(int32_t m) { return (size_t)((m + kScanBlock - 1) / kScanBlock) + 1; }

__global__ void __launch_bounds__(kScanThreads)
scan_blocks_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int32_t m,
                   int32_t* __restrict__ block_sums) {
  __shared__ int s_warp[33];
  const long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  int v[kScanItems];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < m) ? in[base + k] : 0;
    sum += v[k];
  }
  int total;
  int run = block_exclusive_scan(sum, s_warp, total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < m) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
scan_sums_kernel(int32_t* block_sums, int32_t nb, int32_t* out_total) {
  __shared__ int s_warp[33];
  int carry = 0;
  for (int base = 0; base < nb; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const int x = i < nb ? block_sums[i] : 0;
    int total;
    const int r = block_exclusive_scan(x, s_warp, total);
    if (i < nb) block_sums[i] = r + carry;
    carry += total;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

__global__ void scan_add_kernel(int32_t* out, int32_t m, const int32_t* block_sums) {
  const long long i = (long long)blockIdx.x * kScanBlock;
  const int add = block_sums[blockIdx.x];
  for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x)
    if (i + k < m) out[i + k] += add;
}

cudaError_t launch_scan(const int32_t* in, int32_t* out, int32_t m, int32_t* block_sums,
                        cudaStream_t st) {
  const int nb = (m + kScanBlock - 1) / kScanBlock;
  if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), st);
  scan_blocks_kernel<<<nb, kScanThreads, 0, st>>>(in, out, m, block_sums);
  count_launch();
  scan_sums_kernel<<<1, kScanThreads, 0, st>>>(block_sums, nb, out + m);
  count_launch();
  scan_add_kernel<<<nb, 256, 0, st>>>(out, m, block_sums);
  count_launch();
  return cudaGetLastError();
}

// ---- merge: CSR u pairs ---------------------------------------------------------

__global__ void merge_degree_kernel(const int32_t* __restrict__ rp, int32_t n, int32_t* deg) {
  F2M_GRID_STRIDE(v, n) deg[v] = rp[v + 1] - rp[v];
}

__global__ void merge_count_kernel(const int2* __restrict__ pairs, long long npairs, int32_t n,
                                   int32_t* deg, CheckCtl* ctl) {
  F2M_GRID_STRIDE(k, npairs) {
    const int2 p = pairs[k];
    if (p.x < 0 || p.y < 0 || p.x >= n || p.y >= n || p.x == p.y) {
      flag(ctl, kBadPair, k);
      continue;
    }
    atomicAdd(&deg[p.x], 1);
    atomicAdd(&deg[p.y], 1);
  }
}

cudaError_t launch_merge_count(const int32_t* rp, const int2* pairs, int64_t npairs, int32_t n,
                               MergeBuffers& mb, cudaStream_t st) {
  merge_degree_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp, n, mb.deg);
  count_launch();
  if (npairs > 0) {
    merge_count_kernel<<<grid_for(npairs, 256), 256, 0, st>>>(pairs, npairs, n, mb.deg, mb.ctl);
    count_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_scan(mb.deg, mb.tmp_rp, n, mb.block_sums, st);
}

// Rows are strictly increasing (checked when the graph is created, and kept
// so by every merge), so a row that no pair touches comes out of the merge as
// it went in: only the touched rows (those that gained room in tmp_rp) are
// copied, sorted and deduplicated in tmp_col; the others keep their entries.
__device__ __forceinline__ bool merge_touched(const int32_t* rp, const int32_t* tmp_rp, int v) {
  return tmp_rp[v + 1] - tmp_rp[v] != rp[v + 1] - rp[v];
}

// copy a touched row's old entries to the front of its new row; deg becomes
// the append cursor
__global__ void merge_copy_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                  int32_t n, const int32_t* __restrict__ tmp_rp, int32_t* tmp_col,
                                  int32_t* cursor) {
  F2M_GRID_STRIDE(v, n) {
    if (!merge_touched(rp, tmp_rp, (int)v)) continue;
    const int a = rp[v], b = rp[v + 1], o = tmp_rp[v];
    for (int e = a; e < b; ++e) tmp_col[o + (e - a)] = ec[e].x;
    cursor[v] = o + (b - a);
  }
}

__global__ void merge_scatter_kernel(const int2* __restrict__ pairs, long long npairs, int32_t n,
                                     int32_t* tmp_col, int32_t* cursor) {
  F2M_GRID_STRIDE(k, npairs) {
    const int2 p = pairs[k];
    if (p.x < 0 || p.y < 0 || p.x >= n || p.y >= n || p.x == p.y) continue;
    tmp_col[atomicAdd(&cursor[p.x], 1)] = p.y;
    tmp_col[atomicAdd(&cursor[p.y], 1)] = p.x;
  }
}

cudaError_t launch_merge_fill(const int32_t* rp, const int2* ec, const int2* pairs, int64_t npairs,
                              int32_t n, MergeBuffers& mb, cudaStream_t st) {
  merge_copy_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp, ec, n, mb.tmp_rp, mb.tmp_col, mb.deg);
  count_launch();
  if (npairs > 0) {
    merge_scatter_kernel<<<grid_for(npairs, 256), 256, 0, st>>>(pairs, npairs, n, mb.tmp_col,
                                                                mb.deg);
    count_launch();
  }
  return cudaGetLastError();
}

// sort each touched row (insertion sort: rows are short) and count distinct
// columns; an untouched row keeps its length
__global__ void merge_sort_rows_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ tmp_rp,
                                       int32_t* tmp_col, int32_t n, int32_t* uniq) {
  F2M_GRID_STRIDE(v, n) {
    const int a = tmp_rp[v], b = tmp_rp[v + 1];
    if (!merge_touched(rp, tmp_rp, (int)v)) {
      uniq[v] = b - a;
      continue;
    }
    for (int i = a + 1; i < b; ++i) {
      const int x = tmp_col[i];
      int j = i - 1;
      while (j >= a && tmp_col[j] > x) { tmp_col[j + 1] = tmp_col[j]; --j; }
      tmp_col[j + 1] = x;
    }
    int u = 0;
    for (int i = a; i < b; ++i) u += (i == a || tmp_col[i] != tmp_col[i - 1]);
    uniq[v] = u;
  }
}

// the merged rows into ec_out (another array than ec_in): an untouched row's
// entries as they were (its costs are the exact costs of its points), a
// touched row's distinct columns with their exact costs
__global__ void merge_compact_kernel(const int2* __restrict__ xy, const int32_t* __restrict__ rp,
                                     const int2* __restrict__ ec_in, const int32_t* __restrict__ tmp_rp,
                                     const int32_t* __restrict__ tmp_col, int32_t n,
                                     const int32_t* __restrict__ new_rp, int2* __restrict__ ec_out) {
  F2M_GRID_STRIDE(v, n) {
    int o = new_rp[v];
    if (!merge_touched(rp, tmp_rp, (int)v)) {
      for (int e = rp[v]; e < rp[v + 1]; ++e) ec_out[o++] = ec_in[e];
      continue;
    }
    const int a = tmp_rp[v], b = tmp_rp[v + 1];
    const int2 pv = xy[v];
    for (int i = a; i < b; ++i) {
      if (i > a && tmp_col[i] == tmp_col[i - 1]) continue;
      const int c = tmp_col[i];
      ec_out[o++] = make_int2(c, exact_cost(pv, xy[c]));
    }
  }
}

cudaError_t launch_merge_finish(const int2* xy, const int32_t* rp, const int2* ec_in, int32_t n,
                                MergeBuffers& mb, int2* ec_out, cudaStream_t st) {
  merge_sort_rows_kernel<<<grid_for(n, 128), 128, 0, st>>>(rp, mb.tmp_rp, mb.tmp_col, n, mb.deg);
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  err = launch_scan(mb.deg, mb.new_rp, n, mb.block_sums, st);
  if (err != cudaSuccess) return err;
  merge_compact_kernel<<<grid_for(n, 128), 128, 0, st>>>(xy, rp, ec_in, mb.tmp_rp, mb.tmp_col, n, mb.new_rp,
                                                         ec_out);
  count_launch();
  return cudaGetLastError();
}

__global__ void split_ec_kernel(const int2* __restrict__ ec, long long nnz, int32_t* col,
                                int32_t* cost) {
  F2M_GRID_STRIDE(e, nnz) {
    const int2 q = ec[e];
    if (col) col[e] = q.x;
    if (cost) cost[e] = q.y;
  }
}

cudaError_t launch_split_ec(const int2* ec, int64_t nnz, int32_t* col, int32_t* cost,
                            cudaStream_t st) {
  if (nnz == 0) return cudaSuccess;
  split_ec_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(ec, nnz, col, cost);
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
