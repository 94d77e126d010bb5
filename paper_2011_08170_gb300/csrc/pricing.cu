// Pricing scan: every pair u < v outside the candidate CSR with
//   z_uv = c_uv * 2^fb - lambda_u - lambda_v < 0.
// The paper solves on a top-N nearest-neighbour graph and notes that it can
// miss optimal edges (Section 5.3); this scan finds every such edge so the
// final duals are feasible for the complete graph.
//
// N-body tiling: the host lists tile pairs (TILE x TILE blocks of the pair
// triangle of each segment, i.e. instance), handed out by an atomic counter; a CTA keeps TILE j-points in shared memory
// and each thread P i-points in registers.  Per pair an fp32 filter runs:
//   t = s_u + s_v,   e = dy^2 + (dx^2 - t^2)   (two FMAs),   pass if e < 1,
// with s_v = max(lambda_v * 2^-fb + 1/4, 0) * (1 + 2^-19).
// No false negatives: z < 0 implies c < T = (lambda_u + lambda_v) 2^-fb, hence
// sqrt(d2) < c + 1/2 < T + 1/2 <= r_u + r_v with r = max(lambda 2^-fb + 1/4, 0).
// The rounding of r, s and t is below 2^-22 relative, so t >= (r_u + r_v)
// (1 + 2^-20) and t^2 exceeds d2 by more than 2^-20 t^2, while the two FMAs
// err by at most 2^-23 t^2; d2 < 1 (duplicate points) passes trivially.  Pairs
// that pass are decided exactly in integers (exact cost, int64 z), then
// checked against the CSR row by binary search, then appended.
#include <climits>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

constexpr int kPriceThreads = 256;
constexpr int kPriceP = 4;
constexpr int kPriceTile = kPriceThreads * kPriceP;
static_assert(kPriceTile == kPricingTile, "tile size shared with the tile-list builder");

// pts[v] = {x, y, s, node} of node perm[v] (perm NULL: node v); the node id is
// carried in the last component's bits
__global__ void pricing_prep_kernel(const int2* __restrict__ xy, const int32_t* __restrict__ lam,
                                    const int32_t* __restrict__ perm, int32_t n, int32_t fb,
                                    float4* __restrict__ pts) {
  const float scale = ldexpf(1.0f, -fb);
  const float grow = 1.0f + ldexpf(1.0f, -19);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int u = perm ? perm[v] : (int)v;
    const int2 p = xy[u];
    float r = fmaxf((float)lam[u] * scale + 0.25f, 0.0f);
    pts[v] = make_float4((float)p.x, (float)p.y, r * grow, __int_as_float(u));
  }
}

// bounding box and largest s of each listed point range: {min x, min y, max x, max y}, s
__global__ void pricing_boxes_kernel(const float4* __restrict__ pts, const int2* __restrict__ ranges,
                                     float4* __restrict__ box, float* __restrict__ smax) {
  const int2 rg = ranges[blockIdx.x];
  float x0 = 3e38f, y0 = 3e38f, x1 = -3e38f, y1 = -3e38f, sm = 0.f;
  for (int i = rg.x + threadIdx.x; i < rg.y; i += blockDim.x) {
    const float4 q = pts[i];
    x0 = fminf(x0, q.x);
    y0 = fminf(y0, q.y);
    x1 = fmaxf(x1, q.x);
    y1 = fmaxf(y1, q.y);
    sm = fmaxf(sm, q.z);
  }
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
  }
  __shared__ float4 sb[32];
  __shared__ float ss[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sb[warp] = make_float4(x0, y0, x1, y1);
    ss[warp] = sm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 b = sb[0];
    float m = ss[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      b.x = fminf(b.x, sb[w].x);
      b.y = fminf(b.y, sb[w].y);
      b.z = fmaxf(b.z, sb[w].z);
      b.w = fmaxf(b.w, sb[w].w);
      m = fmaxf(m, ss[w]);
    }
    box[blockIdx.x] = b;
    smax[blockIdx.x] = m;
  }
}

// exact decision for a pair that passed the filter: positions ii < jj in the
// point array (each unordered pair once), nodes i and j
__device__ __noinline__ void pricing_confirm(int ii, int jj, int i, int j, int32_t n, const int2* __restrict__ xy,
                                             const int32_t* __restrict__ lam,
                                             const int32_t* __restrict__ rp,
                                             const int2* __restrict__ ec, int32_t fb, int2* pairs,
                                             long long cap, unsigned long long* count) {
  if (jj <= ii || jj >= n) return;  // each unordered pair once; tail of the last tile
  if (j < i) {
    const int t = i;
    i = j;
    j = t;
  }
  const long long S = (long long)lam[i] + lam[j];
  if (S <= 0) return;
  const long long c = exact_cost(xy[i], xy[j]);
  if ((c << fb) - S >= 0) return;
  int lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int cm = ec[mid].x;
    if (cm == j) return;  // already a candidate edge
    if (cm < j) lo = mid + 1; else hi = mid - 1;
  }
  const unsigned long long k = atomicAdd(count, 1ull);
  if ((long long)k < cap) pairs[k] = make_int2(i, j);
}

__global__ void __launch_bounds__(kPriceThreads)
pricing_kernel(const float4* __restrict__ pts, const int2* __restrict__ xy,
               const int32_t* __restrict__ lam, const int32_t* __restrict__ rp,
               const int2* __restrict__ ec, int32_t n, int32_t fb, const int4* __restrict__ tiles,
               int32_t ntiles, int2* pairs, long long cap, unsigned long long* count,
               unsigned int* tile_counter) {
  __shared__ float4 sj[kPriceTile];
  __shared__ int s_tp;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tp = (int)atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int tp = s_tp;
    if (tp >= ntiles) break;
    const int4 tl = tiles[tp];  // i in [x, y), j in [z, w)

    float xi[kPriceP], yi[kPriceP], si[kPriceP];
    int ni[kPriceP];
#pragma unroll
    for (int p = 0; p < kPriceP; ++p) {
      const int i = tl.x + p * kPriceThreads + threadIdx.x;
      if (i < tl.y) {
        const float4 q = pts[i];
        xi[p] = q.x; yi[p] = q.y; si[p] = q.z; ni[p] = __float_as_int(q.w);
      } else {
        xi[p] = 1e18f; yi[p] = 1e18f; si[p] = 0.0f; ni[p] = 0;
      }
    }
    for (int k = threadIdx.x; k < kPriceTile; k += kPriceThreads) {
      const int j = tl.z + k;
      sj[k] = j < tl.w ? pts[j] : make_float4(-1e18f, -1e18f, 0.0f, __int_as_float(0));
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kPriceTile; ++k) {
      const float4 q = sj[k];
      float e[kPriceP];
#pragma unroll
      for (int p = 0; p < kPriceP; ++p) {
        const float dx = q.x - xi[p], dy = q.y - yi[p], t = q.z + si[p];
        e[p] = fmaf(dy, dy, fmaf(dx, dx, -t * t));
      }
      float m = e[0];
#pragma unroll
      for (int p = 1; p < kPriceP; ++p) m = fminf(m, e[p]);
      if (m < 1.0f) {
        const int j = tl.z + k;
#pragma unroll
        for (int p = 0; p < kPriceP; ++p)
          if (e[p] < 1.0f)
            pricing_confirm(tl.x + p * kPriceThreads + threadIdx.x, j, ni[p], __float_as_int(q.w),
                            min(n, tl.w), xy, lam, rp, ec, fb, pairs, cap, count);
      }
    }
  }
}

cudaError_t launch_pricing_prep(const int2* xy, const int32_t* lam, const int32_t* perm, int32_t n, int32_t fb,
                                float4* pts, cudaStream_t st) {
  const int threads = 256;
  int blocks = (int)((n + threads - 1) / threads);
  if (blocks > 4096) blocks = 4096;
  pricing_prep_kernel<<<blocks, threads, 0, st>>>(xy, lam, perm, n, fb, pts);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pricing_boxes(const float4* pts, const int2* ranges, int32_t nranges, float4* box, float* smax,
                                 cudaStream_t st) {
  if (nranges <= 0) return cudaSuccess;
  pricing_boxes_kernel<<<nranges, 256, 0, st>>>(pts, ranges, box, smax);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pricing_scan(const float4* pts, const int2* xy, const int32_t* lam, const int32_t* rp,
                                const int2* ec, int32_t n, int32_t fb, const int4* tiles, int32_t ntiles,
                                int2* pairs, int64_t cap, unsigned long long* count, unsigned int* tile_counter,
                                int num_sms, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(tile_counter, 0, sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (ntiles == 0) return cudaSuccess;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pricing_kernel, kPriceThreads, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)num_sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  pricing_kernel<<<(int)grid, kPriceThreads, 0, st>>>(pts, xy, lam, rp, ec, n, fb, tiles, ntiles,
                                                      pairs, cap, count, tile_counter);
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
