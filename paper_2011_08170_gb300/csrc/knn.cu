// Exact k nearest neighbours on a uniform cell grid: the candidate graph of
// Section 5.3 (each node keeps its top-N nearest neighbours) and the features of
// the learned warm start (distances to the 16 nearest neighbours).
//
// Points are bucketed into square cells of side 2^shift (cell id = row-major
// over a 2^g x 2^g grid covering [0, 2^20)^2) by a radix sort of the cell ids,
// so the points of one cell -- and of a run of cells in one grid row -- are
// contiguous.  One thread per point (in cell order, so a warp's queries are
// neighbours) scans square rings of cells around its own cell, keeps the k best
// (d^2, index) pairs in registers, ordered by exact int64 d^2 then index, and
// stops once the k-th kept d^2 is below the squared distance to the nearest
// cell not yet scanned.  The result is the exact k-NN list with ties broken by
// the smaller index.
#include <climits>

#include <cub/cub.cuh>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

namespace {

__global__ void knn_keys_kernel(const int2* __restrict__ xy, int32_t n, int shift, int gbits,
                                uint64_t* __restrict__ keys, int32_t* __restrict__ idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int2 p = xy[i];
  keys[i] = ((uint64_t)(p.y >> shift) << gbits) | (uint64_t)(p.x >> shift);
  idx[i] = i;
}

__global__ void knn_gather_kernel(const int2* __restrict__ xy, const int32_t* __restrict__ sidx,
                                  int32_t n, int2* __restrict__ sxy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) sxy[i] = xy[sidx[i]];
}

// start[c] = first sorted position whose cell id is >= c, for c in [0, ncell]
__global__ void knn_cell_start_kernel(const uint64_t* __restrict__ skeys, int32_t n, int32_t ncell,
                                      int32_t* __restrict__ start) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > ncell) return;
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (skeys[mid] < (uint64_t)c) lo = mid + 1; else hi = mid;
  }
  start[c] = lo;
}

__device__ __forceinline__ bool knn_less(long long d, int j, long long bd, int bj) {
  return d < bd || (d == bd && j < bj);
}

// Keep the K best (d, j) in ascending order; entries past the k the caller
// asked for are kept too (they never displace a better one).
template <int K>
__device__ __forceinline__ void knn_insert(long long d, int j, long long (&bd)[K], int (&bj)[K]) {
  if (!knn_less(d, j, bd[K - 1], bj[K - 1])) return;
  // entries that (d, j) precedes move up one place; it lands after the last
  // entry that precedes it
#pragma unroll
  for (int p = K - 1; p > 0; --p) {
    if (knn_less(d, j, bd[p], bj[p])) {
      if (knn_less(d, j, bd[p - 1], bj[p - 1])) {
        bd[p] = bd[p - 1];
        bj[p] = bj[p - 1];
      } else {
        bd[p] = d;
        bj[p] = j;
      }
    }
  }
  if (knn_less(d, j, bd[0], bj[0])) {
    bd[0] = d;
    bj[0] = j;
  }
}

template <int K>
__device__ __forceinline__ void knn_scan(const int2* __restrict__ sxy, const int32_t* __restrict__ sidx,
                                         int a, int b, int self, int x, int y, long long (&bd)[K],
                                         int (&bj)[K]) {
  for (int p = a; p < b; ++p) {
    if (p == self) continue;
    const int2 q = sxy[p];
    const long long dx = (long long)q.x - x, dy = (long long)q.y - y;
    knn_insert<K>(dx * dx + dy * dy, sidx[p], bd, bj);
  }
}

template <int K>
__global__ void __launch_bounds__(128)
knn_query_kernel(const int2* __restrict__ sxy, const int32_t* __restrict__ sidx,
                 const int32_t* __restrict__ start, int32_t n, int32_t k, int shift, int gbits,
                 int32_t* __restrict__ nbr, long long* __restrict__ d2out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int2 me = sxy[t];
  const int x = me.x, y = me.y;
  const int gdim = 1 << gbits;
  const int cx = x >> shift, cy = y >> shift;
  long long bd[K];
  int bj[K];
#pragma unroll
  for (int p = 0; p < K; ++p) {
    bd[p] = LLONG_MAX;
    bj[p] = INT_MAX;
  }
  for (int r = 0;; ++r) {
    const int x0 = cx - r, x1 = cx + r, y0 = cy - r, y1 = cy + r;
    const int ya = max(y0, 0), yb = min(y1, gdim - 1);
    const int xa = max(x0, 0), xb = min(x1, gdim - 1);
    for (int gy = ya; gy <= yb; ++gy) {
      const int row = gy << gbits;
      // a full row of the ring is one contiguous run of cells; other rows
      // contribute the cells at x0 and x1
      const bool full = (gy == y0 || gy == y1);
      int a0, b0, a1 = 0, b1 = 0;
      if (full) {
        a0 = start[row + xa];
        b0 = start[row + xb + 1];
      } else {
        a0 = x0 >= 0 ? start[row + x0] : 0;
        b0 = x0 >= 0 ? start[row + x0 + 1] : 0;
        if (x1 < gdim && x1 != x0) {
          a1 = start[row + x1];
          b1 = start[row + x1 + 1];
        }
      }
      for (int part = 0; part < 2; ++part) {
        const int a = part ? a1 : a0, b = part ? b1 : b0;
        knn_scan<K>(sxy, sidx, a, b, t, x, y, bd, bj);
      }
    }
    // smallest distance from (x, y) to a cell outside the scanned square
    long long bnd = LLONG_MAX;
    if (x0 > 0) bnd = min(bnd, (long long)x - ((long long)x0 << shift) + 1);
    if (y0 > 0) bnd = min(bnd, (long long)y - ((long long)y0 << shift) + 1);
    if (x1 < gdim - 1) bnd = min(bnd, ((long long)(x1 + 1) << shift) - x);
    if (y1 < gdim - 1) bnd = min(bnd, ((long long)(y1 + 1) << shift) - y);
    if (bnd == LLONG_MAX) break;  // the whole grid has been scanned
    long long kth = LLONG_MAX;
#pragma unroll
    for (int p = 0; p < K; ++p)
      if (p == k - 1) kth = bd[p];
    if (kth < bnd * bnd) break;
  }
  const int q = sidx[t];
#pragma unroll
  for (int p = 0; p < K; ++p) {
    if (p < k) {
      nbr[(size_t)q * k + p] = bj[p];
      if (d2out) d2out[(size_t)q * k + p] = bd[p];
    }
  }
}

// symmetrised pair keys (u << 32 | w) of both directions of every k-NN entry
__global__ void knn_pair_keys_kernel(const int32_t* __restrict__ nbr, int32_t n, int32_t k,
                                     uint64_t* __restrict__ keys) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long m = (long long)n * k;
  if (e >= m) return;
  const uint64_t u = (uint64_t)(e / k), w = (uint64_t)(uint32_t)nbr[e];
  keys[2 * e] = (u << 32) | w;
  keys[2 * e + 1] = (w << 32) | u;
}

__global__ void knn_csr_rows_kernel(const uint64_t* __restrict__ ukeys, const int* __restrict__ d_nnz,
                                    int32_t n, int32_t* __restrict__ row_ptr) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v > n) return;
  int lo = 0, hi = *d_nnz;
  const uint64_t key = (uint64_t)v << 32;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ukeys[mid] < key) lo = mid + 1; else hi = mid;
  }
  row_ptr[v] = lo;
}

__global__ void knn_csr_cols_kernel(const uint64_t* __restrict__ ukeys, const int* __restrict__ d_nnz,
                                    int32_t* __restrict__ col) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < *d_nnz) col[e] = (int32_t)(uint32_t)(ukeys[e] & 0xffffffffu);
}

__global__ void features_kernel(const long long* __restrict__ d2, int32_t n, float* __restrict__ feat,
                                float* __restrict__ scale) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double dist[kFeatures];
  double sum = 0.0;
#pragma unroll
  for (int j = 0; j < kFeatures; ++j) {
    dist[j] = sqrt((double)d2[(size_t)v * kFeatures + j]);
    sum += dist[j];
  }
  const double s = fmax(1.0, sum / kFeatures);
#pragma unroll
  for (int j = 0; j < kFeatures; ++j) feat[(size_t)v * kFeatures + j] = (float)(dist[j] / s);
  scale[v] = (float)s;
}

inline unsigned blocks_for(long long items, int threads) {
  return (unsigned)((items + threads - 1) / threads);
}

}  // namespace

// grid: the smallest g with 4^g >= n / 2 (about 2 points per cell when the
// points fill the square), cells of side 2^(20 - g)
static void knn_grid(int32_t n, int* shift, int* gbits) {
  int g = 1;
  while (g < 11 && (1LL << (2 * g)) < (long long)n / 2) ++g;
  *gbits = g;
  *shift = 20 - g;
}

cudaError_t knn_device(const int2* d_xy, int32_t n, int32_t k, int32_t* d_nbr, long long* d_d2,
                       cudaStream_t st) {
  if (k < 1 || k > kKnnMax || n <= k) return cudaErrorInvalidValue;
  int shift = 0, gbits = 0;
  knn_grid(n, &shift, &gbits);
  const int ncell = 1 << (2 * gbits);
  uint64_t *keys = nullptr, *skeys = nullptr;
  int32_t *idx = nullptr, *sidx = nullptr, *start = nullptr;
  int2* sxy = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  cudaError_t e = sort_pairs_u64(nullptr, tmp_bytes, nullptr, nullptr, nullptr, nullptr, n, 2 * gbits, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&keys, sizeof(uint64_t) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&skeys, sizeof(uint64_t) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&idx, sizeof(int32_t) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&sidx, sizeof(int32_t) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&start, sizeof(int32_t) * (ncell + 1), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&sxy, sizeof(int2) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&tmp, tmp_bytes ? tmp_bytes : 1, st);
  if (e == cudaSuccess) {
    knn_keys_kernel<<<blocks_for(n, 256), 256, 0, st>>>(d_xy, n, shift, gbits, keys, idx);
    count_launch();
    e = sort_pairs_u64(tmp, tmp_bytes, keys, skeys, idx, sidx, n, 2 * gbits, st);
  }
  if (e == cudaSuccess) {
    knn_gather_kernel<<<blocks_for(n, 256), 256, 0, st>>>(d_xy, sidx, n, sxy);
    count_launch();
    knn_cell_start_kernel<<<blocks_for(ncell + 1, 256), 256, 0, st>>>(skeys, n, ncell, start);
    count_launch();
    const unsigned nb = blocks_for(n, 128);
    if (k <= 8)
      knn_query_kernel<8><<<nb, 128, 0, st>>>(sxy, sidx, start, n, k, shift, gbits, d_nbr, d_d2);
    else if (k <= 16)
      knn_query_kernel<16><<<nb, 128, 0, st>>>(sxy, sidx, start, n, k, shift, gbits, d_nbr, d_d2);
    else
      knn_query_kernel<32><<<nb, 128, 0, st>>>(sxy, sidx, start, n, k, shift, gbits, d_nbr, d_d2);
    count_launch();
    e = cudaGetLastError();
  }
  cudaFreeAsync(keys, st);
  cudaFreeAsync(skeys, st);
  cudaFreeAsync(idx, st);
  cudaFreeAsync(sidx, st);
  cudaFreeAsync(start, st);
  cudaFreeAsync(sxy, st);
  cudaFreeAsync(tmp, st);
  return e;
}

cudaError_t knn_csr_device(const int2* d_xy, int32_t n, int32_t k, int32_t* d_row_ptr, int32_t* d_col,
                           int64_t* nnz_out, cudaStream_t st) {
  const long long m = 2LL * n * k;
  if (m >= INT_MAX) return cudaErrorInvalidValue;
  int32_t* nbr = nullptr;
  uint64_t *keys = nullptr, *skeys = nullptr, *ukeys = nullptr;
  int* d_nnz = nullptr;
  void* tmp = nullptr;
  size_t sort_bytes = 0, uniq_bytes = 0;
  cudaError_t e = cub::DeviceRadixSort::SortKeys(nullptr, sort_bytes, (const uint64_t*)nullptr,
                                                 (uint64_t*)nullptr, (int)m, 0, 64, st);
  if (e == cudaSuccess)
    e = cub::DeviceSelect::Unique(nullptr, uniq_bytes, (const uint64_t*)nullptr, (uint64_t*)nullptr,
                                  (int*)nullptr, (int)m, st);
  const size_t tmp_bytes = sort_bytes > uniq_bytes ? sort_bytes : uniq_bytes;
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&nbr, sizeof(int32_t) * n * (size_t)k, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&keys, sizeof(uint64_t) * m, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&skeys, sizeof(uint64_t) * m, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&ukeys, sizeof(uint64_t) * m, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_nnz, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&tmp, tmp_bytes ? tmp_bytes : 1, st);
  if (e == cudaSuccess) e = knn_device(d_xy, n, k, nbr, nullptr, st);
  if (e == cudaSuccess) {
    knn_pair_keys_kernel<<<blocks_for((long long)n * k, 256), 256, 0, st>>>(nbr, n, k, keys);
    count_launch();
    size_t b = tmp_bytes;
    e = cub::DeviceRadixSort::SortKeys(tmp, b, keys, skeys, (int)m, 0, 64, st);
  }
  if (e == cudaSuccess) {
    size_t b = tmp_bytes;
    e = cub::DeviceSelect::Unique(tmp, b, skeys, ukeys, d_nnz, (int)m, st);
  }
  if (e == cudaSuccess) {
    knn_csr_rows_kernel<<<blocks_for(n + 1, 256), 256, 0, st>>>(ukeys, d_nnz, n, d_row_ptr);
    count_launch();
    knn_csr_cols_kernel<<<blocks_for(m, 256), 256, 0, st>>>(ukeys, d_nnz, d_col);
    count_launch();
    e = cudaGetLastError();
  }
  int h_nnz = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_nnz, d_nnz, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *nnz_out = h_nnz;
  cudaFreeAsync(nbr, st);
  cudaFreeAsync(keys, st);
  cudaFreeAsync(skeys, st);
  cudaFreeAsync(ukeys, st);
  cudaFreeAsync(d_nnz, st);
  cudaFreeAsync(tmp, st);
  return e;
}

cudaError_t features_device(const int2* d_xy, int32_t n, float* d_feat, float* d_scale,
                            cudaStream_t st) {
  long long* d2 = nullptr;
  int32_t* nbr = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d2, sizeof(long long) * n * (size_t)kFeatures, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&nbr, sizeof(int32_t) * n * (size_t)kFeatures, st);
  if (e == cudaSuccess) e = knn_device(d_xy, n, kFeatures, nbr, d2, st);
  if (e == cudaSuccess) {
    features_kernel<<<blocks_for(n, 128), 128, 0, st>>>(d2, n, d_feat, d_scale);
    count_launch();
    e = cudaGetLastError();
  }
  cudaFreeAsync(d2, st);
  cudaFreeAsync(nbr, st);
  return e;
}

}  // namespace f2m
