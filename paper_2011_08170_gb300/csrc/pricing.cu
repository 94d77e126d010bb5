// Pricing scan: every pair u < v outside the candidate CSR with
//   z_uv = c_uv * 2^fb - lambda_u - lambda_v < 0.
// The paper solves on a top-N nearest-neighbour graph and notes that it can
// miss optimal edges (Section 5.3); this scan finds every such edge so the
// final duals are feasible for the complete graph.
//
// N-body tiling: the host lists tile pairs (blocks of the pair triangle of
// each segment, i.e. instance: up to kPricingTile i-points by up to
// kPricingTile j-points; the scan's lists use kPricingJ j-points, so the last
// wave of tile pairs is short), handed out by an atomic counter; a CTA keeps
// the j-points in shared memory and each thread P i-points in registers, two
// at a time in packed fp32x2 registers (Blackwell's two-lane FADD2 / FFMA2:
// one issue slot for two pairs).
//
// Filter.  r_v = max(lambda_v 2^-fb + 1/4, 0), s_v = (r_v + 2)(1 + 2^-17) in
// fp32, a_v = x_v - s_v, c_v = x_v + s_v.  Per pair, with t = s_u + s_v:
//   u = a_v - c_u = dx - t,  w = c_v - a_u = dx + t,  dy = y_v - y_u,
//   e' = dy^2 + (u w - 1) = d^2 - t^2 - 1      (3 FADD2 + 2 FFMA2 per 2 pairs)
// and the pair passes when e' < 0.  The sign bits are OR-ed over a thread's
// pairs with 4 j-points; a warp appends the groups with a set bit to its list
// in shared memory (ballot, no atomics) and, after every 64 j-points, its
// lanes re-evaluate the listed pairs and decide the passing ones exactly, so
// the hot loop holds no call and no block-wide barrier.  No false negatives: z < 0 implies c < T = (lambda_u + lambda_v)
// 2^-fb, hence d < c + 1/2 < T + 1/2 <= R = r_u + r_v, and t >= (R + 4)(1 +
// 2^-17.3) after the roundings of r (2^-23 relative) and s, so d^2 - t^2 <=
// -(4 + 2^-17.3 t)(t + d).  The fp32 errors are at most 0.5 (t + d) (a, c and
// u, w: 2^-24 of |x| + s < 2^20 + s each) plus 2^-20.9 t (t + d) (the products
// and the sum), so e' stays negative.  Pairs that pass are decided exactly in
// integers (exact cost, int64 z), then checked against the CSR row by binary
// search, then appended.
#include <climits>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

// A CTA takes kPricingTile i-points (P per thread, as P / 2 packed pairs) and
// kPricingTile j-points.  P = 8 (128 threads) when there are many tile pairs,
// P = 4 (256 threads: twice the threads on one tile pair) when there are few.
constexpr int kPriceTile = kPricingTile;
constexpr int kPriceJMax = kPricingJ;  // j-points of a tile pair: the scan's lists never hold more

// pts[v] = {x, y, s, node} of node perm[v] (perm NULL: node v); the node id is
// carried in the last component's bits
__global__ void pricing_prep_kernel(const int2* __restrict__ xy, const int32_t* __restrict__ lam,
                                    const int32_t* __restrict__ perm, int32_t n, int32_t fb,
                                    float4* __restrict__ pts) {
  const float scale = ldexpf(1.0f, -fb);
  const float grow = 1.0f + ldexpf(1.0f, -17);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int u = perm ? perm[v] : (int)v;
    const int2 p = xy[u];
    const float r = fmaxf((float)lam[u] * scale + 0.25f, 0.0f);
    pts[v] = make_float4((float)p.x, (float)p.y, (r + 2.0f) * grow, __int_as_float(u));
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

// The filter of one pair, from a_v, c_v, y_v of the j-point and the negated
// a_u, c_u, y_u of the i-point; the hot loop evaluates the same operations two
// pairs at a time
__device__ __forceinline__ float pricing_filter(float aj, float cj, float yj, float nai, float nci, float nyi) {
  const float u = __fadd_rn(aj, nci), w = __fadd_rn(cj, nai), dy = __fadd_rn(yj, nyi);
  return __fmaf_rn(dy, dy, __fmaf_rn(u, w, -1.0f));
}

// j-points per sign test, and per chunk after which a warp decides its hits;
// a warp's list holds one chunk (one entry per lane and group at most)
constexpr int kPriceGroup = 4;
constexpr int kPriceChunk = 64;
constexpr int kWarpHits = (kPriceChunk / kPriceGroup) * 32;
static_assert(kPriceJMax % kPriceChunk == 0 && kPriceChunk % kPriceGroup == 0, "chunking");

// Decide exactly every passing pair of the groups in a warp's hit list (each
// entry: first j of the group << 8 | thread); all lanes of the warp take part.
template <int P>
__device__ __forceinline__ void pricing_hits(const int* hits, int nh, int lane, int4 tl, const float4* s_ac,
                                          const float2* s_y, const float4* __restrict__ pts,
                                          const int2* __restrict__ xy, const int32_t* __restrict__ lam,
                                          const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                          int32_t n, int32_t fb, int2* pairs, long long cap,
                                          unsigned long long* count) {
  constexpr int kPriceThreads = kPriceTile / P;
  for (int h = lane; h < nh * P; h += 32) {
    const int ent = hits[h / P], p = h % P;
    const int t = ent & 0xFF, g = ent >> 8;
    const int ii = tl.x + p * kPriceThreads + t;
    if (ii >= tl.y) continue;
    const float4 vi = pts[ii];
    const float nai = -(vi.x - vi.z), nci = -(vi.x + vi.z), nyi = -vi.y;
    for (int kk = 0; kk < kPriceGroup; ++kk) {
      const int jj = tl.z + g + kk;
      if (jj >= tl.w) break;
      const float4 ac = s_ac[g + kk];
      if (pricing_filter(ac.x, ac.z, s_y[g + kk].x, nai, nci, nyi) < 0.0f)
        pricing_confirm(ii, jj, __float_as_int(vi.w), __float_as_int(pts[jj].w), min(n, tl.w), xy, lam, rp,
                        ec, fb, pairs, cap, count);
    }
  }
}

template <int P>
__global__ void __launch_bounds__(kPricingTile / P, P == 8 ? 7 : 4)
pricing_kernel(const float4* __restrict__ pts, const int2* __restrict__ xy,
               const int32_t* __restrict__ lam, const int32_t* __restrict__ rp,
               const int2* __restrict__ ec, int32_t n, int32_t fb, const int4* __restrict__ tiles,
               int32_t ntiles, int2* pairs, long long cap, unsigned long long* count,
               unsigned int* tile_counter) {
  constexpr int kPriceThreads = kPriceTile / P;
  constexpr int Q = P / 2;
  static_assert(kPriceThreads <= 256 && kPriceTile <= (1 << 23), "hit entry packing");
  __shared__ float4 s_ac[kPriceJMax];                       // {a, a, c, c} of the j-points
  __shared__ float2 s_y[kPriceJMax];                        // {y, y}
  __shared__ int s_hit[(kPriceThreads / 32) * kWarpHits];  // one list per warp
  __shared__ int s_tp;
  const float2 minus_one = make_float2(-1.0f, -1.0f);
  const int lane = threadIdx.x & 31;
  int* hits = s_hit + (threadIdx.x >> 5) * kWarpHits;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tp = (int)atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int tp = s_tp;
    if (tp >= ntiles) break;
    const int4 tl = tiles[tp];  // i in [x, y), j in [z, w)

    // i-points p = 2q + h at tl.x + p * kPriceThreads + tid, negated; a point
    // past the range gets 1e18 (its e' stays above 1e36, finite)
    float2 na[Q], nc[Q], ny[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float a[2], c[2], y[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = tl.x + (2 * q + h) * kPriceThreads + threadIdx.x;
        if (i < tl.y) {
          const float4 v = pts[i];
          a[h] = v.x - v.z;
          c[h] = v.x + v.z;
          y[h] = v.y;
        } else {
          a[h] = 1e18f;
          c[h] = 1e18f;
          y[h] = 1e18f;
        }
      }
      na[q] = make_float2(-a[0], -a[1]);
      nc[q] = make_float2(-c[0], -c[1]);
      ny[q] = make_float2(-y[0], -y[1]);
    }
    // the tile's j-points, rounded up to whole chunks (at most kPriceTile)
    const int kend = min(kPriceJMax, (tl.w - tl.z + kPriceChunk - 1) / kPriceChunk * kPriceChunk);
    for (int k = threadIdx.x; k < kend; k += kPriceThreads) {
      const int j = tl.z + k;
      if (j < tl.w) {
        const float4 v = pts[j];
        const float a = v.x - v.z, c = v.x + v.z;
        s_ac[k] = make_float4(a, a, c, c);
        s_y[k] = make_float2(v.y, v.y);
      } else {
        s_ac[k] = make_float4(-1e18f, -1e18f, -1e18f, -1e18f);
        s_y[k] = make_float2(-1e18f, -1e18f);
      }
    }
    __syncthreads();
    for (int k0 = 0; k0 < kend; k0 += kPriceChunk) {
      int nh = 0;  // entries in this warp's list (the same in every lane)
#pragma unroll 2
      for (int g = k0; g < k0 + kPriceChunk; g += kPriceGroup) {
        unsigned int sign = 0u;
#pragma unroll
        for (int kk = 0; kk < kPriceGroup; ++kk) {
          const float4 ac = s_ac[g + kk];
          const float2 yj = s_y[g + kk];
          const float2 aj = make_float2(ac.x, ac.y), cj = make_float2(ac.z, ac.w);
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const float2 u = __fadd2_rn(aj, nc[q]);
            const float2 w = __fadd2_rn(cj, na[q]);
            const float2 dy = __fadd2_rn(yj, ny[q]);
            const float2 e = __ffma2_rn(dy, dy, __ffma2_rn(u, w, minus_one));
            sign |= __float_as_uint(e.x) | __float_as_uint(e.y);
          }
        }
        const unsigned int m = __ballot_sync(0xffffffffu, (int)sign < 0);
        if (m) {  // rare: append the lanes' groups to the warp's list
          if ((int)sign < 0) hits[nh + __popc(m & ((1u << lane) - 1u))] = (g << 8) | (int)threadIdx.x;
          nh += __popc(m);
        }
      }
      if (nh) {  // the same branch in every lane of the warp
        __syncwarp();
        pricing_hits<P>(hits, nh, lane, tl, s_ac, s_y, pts, xy, lam, rp, ec, n, fb, pairs, cap, count);
        __syncwarp();  // the list is free for the next chunk
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
  // P = 8 when the tile pairs fill the GPU several times over
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pricing_kernel<8>, kPriceTile / 8, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  if ((long long)ntiles >= 4LL * num_sms * per_sm) {
    const long long grid = (long long)num_sms * per_sm;
    pricing_kernel<8><<<(int)grid, kPriceTile / 8, 0, st>>>(pts, xy, lam, rp, ec, n, fb, tiles, ntiles, pairs,
                                                           cap, count, tile_counter);
  } else {
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pricing_kernel<4>, kPriceTile / 4, 0);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)num_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    pricing_kernel<4><<<(int)grid, kPriceTile / 4, 0, st>>>(pts, xy, lam, rp, ec, n, fb, tiles, ntiles, pairs,
                                                           cap, count, tile_counter);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
