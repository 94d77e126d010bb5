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
#include <cuda_fp16.h>

#include <climits>
#include <cmath>

#include "f2m_device.cuh"
#include "f2m_internal.h"
#include "tcgen05.cuh"

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
// (inU non-NULL: the i-points are the nodes flagged in inU, the j-points all
// nodes; a pair of two flagged nodes is taken from the row of the smaller)
__device__ __noinline__ void pricing_confirm(int ii, int jj, int i, int j, int32_t n, const int2* __restrict__ xy,
                                             const int32_t* __restrict__ lam,
                                             const int32_t* __restrict__ rp,
                                             const int2* __restrict__ ec, int32_t fb, int2* pairs,
                                             long long cap, unsigned long long* count,
                                             const uint8_t* __restrict__ inU = nullptr) {
  if (inU) {
    if (jj >= n || j == i || (inU[j] && j < i)) return;
  } else if (jj <= ii || jj >= n) {
    return;  // each unordered pair once; tail of the last tile
  }
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
                                          const float4* __restrict__ pts_i, const uint8_t* __restrict__ inU,
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
    const float4 vi = pts_i[ii];
    const float nai = -(vi.x - vi.z), nci = -(vi.x + vi.z), nyi = -vi.y;
    for (int kk = 0; kk < kPriceGroup; ++kk) {
      const int jj = tl.z + g + kk;
      if (jj >= tl.w) break;
      const float4 ac = s_ac[g + kk];
      if (pricing_filter(ac.x, ac.z, s_y[g + kk].x, nai, nci, nyi) < 0.0f)
        pricing_confirm(ii, jj, __float_as_int(vi.w), __float_as_int(pts[jj].w), min(n, tl.w), xy, lam, rp,
                        ec, fb, pairs, cap, count, inU);
    }
  }
}

template <int P>
__global__ void __launch_bounds__(kPricingTile / P, P == 8 ? 7 : 4)
pricing_kernel(const float4* __restrict__ pts, const int2* __restrict__ xy,
               const int32_t* __restrict__ lam, const int32_t* __restrict__ rp,
               const int2* __restrict__ ec, int32_t n, int32_t fb, const int4* __restrict__ tiles,
               int32_t ntiles, int2* pairs, long long cap, unsigned long long* count,
               unsigned int* tile_counter, const float4* __restrict__ pts_i, const uint8_t* __restrict__ inU,
               int32_t ni, int32_t nj_tiles) {
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
    // i in [x, y), j in [z, w); no list: i-tiles of the ni i-points by j-tiles of all points
    int4 tl;
    if (tiles) {
      tl = tiles[tp];
    } else {
      const int it = tp / nj_tiles, jt = tp % nj_tiles;
      tl = make_int4(it * kPriceTile, min((it + 1) * kPriceTile, ni), jt * kPriceJMax, min((jt + 1) * kPriceJMax, n));
    }

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
          const float4 v = pts_i[i];
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
        pricing_hits<P>(hits, nh, lane, tl, s_ac, s_y, pts, pts_i, inU, xy, lam, rp, ec, n, fb, pairs, cap, count);
        __syncwarp();  // the list is free for the next chunk
      }
    }
  }
}

// the nodes whose lambda (units 2^-fb) exceeds the reference (units 2^-fb_ref,
// fb >= fb_ref) scaled to fb: flagged in inU, their points appended to pts_u
// (order unspecified), their number in *count
__global__ void pricing_raised_kernel(const int32_t* __restrict__ lam, const int32_t* __restrict__ lam_ref,
                                      int32_t n, int32_t shift, const float4* __restrict__ pts,
                                      uint8_t* __restrict__ inU, float4* __restrict__ pts_u,
                                      unsigned int* count) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const bool up = (long long)lam[v] > ((long long)lam_ref[v] << shift);
    inU[v] = up ? 1 : 0;
    if (up) pts_u[atomicAdd(count, 1u)] = pts[v];
  }
}

cudaError_t launch_pricing_raised(const int32_t* lam, const int32_t* lam_ref, int32_t n, int32_t shift,
                                  const float4* pts, uint8_t* inU, float4* pts_u, unsigned int* count,
                                  cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  pricing_raised_kernel<<<blocks, 256, 0, st>>>(lam, lam_ref, n, shift, pts, inU, pts_u, count);
  count_launch();
  return cudaGetLastError();
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
                                int num_sms, cudaStream_t st, const float4* pts_i, const uint8_t* inU, int32_t ni) {
  if (!pts_i) pts_i = pts;
  const int32_t nj_tiles = (n + kPriceJMax - 1) / kPriceJMax;
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
                                                           cap, count, tile_counter, pts_i, inU, ni, nj_tiles);
  } else {
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pricing_kernel<4>, kPriceTile / 4, 0);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)num_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    pricing_kernel<4><<<(int)grid, kPriceTile / 4, 0, st>>>(pts, xy, lam, rp, ec, n, fb, tiles, ntiles, pairs,
                                                           cap, count, tile_counter, pts_i, inU, ni, nj_tiles);
  }
  count_launch();
  return cudaGetLastError();
}


// ---- The scan on the tensor cores ------------------------------------------------
//
// The same pairs, the same exact decision (pricing_confirm), a different filter:
// for a tile pair of 128 i-points and 256 j-points (positions in the
// renumbered order, where a tile is a compact patch), quantised integer
// coordinates in a frame fitted to the pair turn the test into a small integer
// matrix product that one tcgen05.mma computes exactly.
//
// Frame: (bx0, by0) = the low corner of the pair's bounding box, q = 2^b, b the
// smallest shift with every X = (x - bx0) >> b, Y = (y - by0) >> b in
// [0, 1023] and every radius R below in [0, 1023].  Radius, with m = b + fb:
//   R_u = max(0, ceil((4 lambda_u + 2^fb + C_m) / 2^(m+2))),
//   C_m = ceil(sqrt(2^(2m+3))) >= 2^(m+2) sqrt(2) / 2,
// so R_u >= rho_u = (lambda_u 2^-fb + 1/4) / q + sqrt(2)/2.
// No false negatives: z_uv < 0 means c_uv < T = (lambda_u + lambda_v) 2^-fb,
// so the distance d < c + 1/2 < T + 1/2.  With x - bx0 = q X + f (0 <= f < q)
// the true difference vector is q D + f' with D = (X_u - X_v, Y_u - Y_v) and
// |f'| < sqrt(2) q, so q |D| - sqrt(2) q < d < T + 1/2, i.e.
// |D| < rho_u + rho_v <= R_u + R_v, and e = |D|^2 - (R_u + R_v)^2 < 0.
// Expanded, e = A_u + A_v - 2 (X_u X_v + Y_u Y_v + R_u R_v), A = X^2 + Y^2 - R^2,
// which is the product of the fp16 rows
//   i-point: [A_hi, A_lo, 2048, 1, X, Y, R, 0 ...]      (A = 2048 A_hi + A_lo)
//   j-point: [2048, 1, A_hi, A_lo, -2X, -2Y, -2R, 0 ...]
// Every entry is an integer of at most 11 bits (exact in fp16), every product
// at most 2^21 in magnitude and every partial sum of the seven below 2^24, so
// the fp32 accumulator holds e exactly, whatever the order of the additions.
// A row past the tile's points is [1024, 0, 2048, 1, 0, 0, 0] (a column past
// them [2048, 1, 1024, 0, 0, 0, 0]): e >= 2^21 - 1023^2 > 0, never a candidate.
//
// Per scan, small kernels prepare the points {x, y, lambda, node} in the
// renumbered order, each 128-point block's bounding box and largest lambda,
// and each tile pair's frame {bx0, by0, b, m} from the boxes and lambdas of
// its two blocks.  The scan runs one CTA of 30 warps per SM over a contiguous
// part of the tile-pair list, its warps in roles that hand tile pairs on
// through mbarriers (no CTA barrier in the loop): one warp copies the tile
// entries and frames (64 at a time) and each tile pair's points (bulk copies,
// five stages); 8 warps write the operand rows (one a thread) into one of four
// shared-memory stages; one thread issues the 128 x 128 x 16 MMA into one of
// four 128-column fp32 accumulators in tensor memory and commits it; 16 warps
// read the accumulators (warp w: lanes 32 (w mod 4) .. + 31, 32 columns), OR
// the sign bits three at a time (lop3) and append the negative values, pairs
// u < v inside the tile pair, to a candidate list.  A last kernel decides the
// candidates: the fp32 filter of the CUDA-core scan, then exactly.  Waiting
// threads sleep on the mbarriers (try_wait with a suspend-time hint).

constexpr int kMmaI = kMmaTileI;  // i-points per tile pair (MMA M, TMEM lanes)
constexpr int kMmaJ = kMmaTileJ;  // j-points per tile pair (MMA N, TMEM columns)
static_assert(kMmaI == 128 && kMmaJ == kMmaI, "an i-block and a j-block of 128 points");
constexpr int kMmaAcc = 4;  // accumulators (and operand stages) in flight: 4 x 128 TMEM columns
// warp roles of the scan's CTA: copies, MMA issue, 8 warps writing operand
// rows (one row a thread), 16 warps reading accumulators (4 per TMEM lane
// quarter, 32 columns each); they hand tile pairs on through mbarriers
constexpr int kMmaWarpCopy = 0, kMmaWarpMma = 1, kMmaWarpBuild = 2, kMmaBuildWarps = 8;
constexpr int kMmaWarpEpi = kMmaWarpBuild + kMmaBuildWarps, kMmaEpiWarps = 16;
constexpr int kMmaThreads = 32 * (kMmaWarpEpi + kMmaEpiWarps);
static_assert(kMmaBuildWarps * 32 == kMmaI + kMmaJ, "one operand row a builder thread");
constexpr int kMmaCoordMax = 1023;
constexpr long long kMmaWaitLimit = 1LL << 26;

struct MmaArgs {
  const int4* pts4;        // {x, y, lambda, node} per position
  const int4* tiles;       // {i0, i1, j0, j1} positions
  const int4* frames;      // per tile pair {bx0, by0, b, m}
  int32_t ntiles;
  int32_t fb;
  const int2* xy;
  const int32_t* lam;
  const int32_t* rp;
  const int2* ec;
  int2* pairs;
  long long cap;
  unsigned long long* count;
  unsigned int* tile_counter;
  int32_t* status;         // bit 0: an mbarrier wait gave up
  int2* cand;              // candidate pairs {ii, jj} (positions), decided by pricing_mma_confirm_kernel
  unsigned long long* ncand;
  long long cand_cap;
  long long cm[40];        // C_m = ceil(sqrt(2^(2m+3))), m = b + fb
};

// pts4[v] = {x, y, lambda, node} of node perm[v]
__global__ void pricing_mma_prep_kernel(const int2* __restrict__ xy, const int32_t* __restrict__ lam,
                                        const int32_t* __restrict__ perm, int32_t n, int4* __restrict__ pts4) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int u = perm[v];
    const int2 p = xy[u];
    pts4[v] = make_int4(p.x, p.y, lam[u], u);
  }
}

__device__ __forceinline__ uint32_t mma_pack_h2(int lo, int hi) {
  const __half2 h = __halves2half2(__int2half_rn(lo), __int2half_rn(hi));
  return *reinterpret_cast<const uint32_t*>(&h);
}

// radius of a point in the frame with m = b + fb (see above)
__device__ __forceinline__ int mma_radius(int lam, int fb, int m, long long cm) {
  const long long num = 4LL * lam + (1LL << fb) + cm;
  const long long r = (num + (1LL << (m + 2)) - 1) >> (m + 2);
  return r > 0 ? (int)r : 0;
}

// per 128-point block (ranges [x, y) of positions): bounding box and largest
// lambda; one warp per block
__global__ void pricing_mma_blocks_kernel(const int4* __restrict__ pts4, const int2* __restrict__ ranges,
                                          int32_t nblocks, int4* __restrict__ box, int32_t* __restrict__ lmax) {
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (wid >= nblocks) return;
  const int2 rg = ranges[wid];
  int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN, lm = INT_MIN;
  for (int v = rg.x + lane; v < rg.y; v += 32) {
    const int4 q = pts4[v];
    x0 = min(x0, q.x);
    y0 = min(y0, q.y);
    x1 = max(x1, q.x);
    y1 = max(y1, q.y);
    lm = max(lm, q.z);
  }
  x0 = __reduce_min_sync(0xffffffffu, x0);
  y0 = __reduce_min_sync(0xffffffffu, y0);
  x1 = __reduce_max_sync(0xffffffffu, x1);
  y1 = __reduce_max_sync(0xffffffffu, y1);
  lm = __reduce_max_sync(0xffffffffu, lm);
  if (lane == 0) {
    box[wid] = make_int4(x0, y0, x1, y1);
    lmax[wid] = lm;
  }
}

// per tile pair (its blocks {ib, jb0, jb1 or -1}): the frame {bx0, by0, b, m}
__global__ void pricing_mma_frames_kernel(const int4* __restrict__ tblk, int32_t ntiles,
                                          const int4* __restrict__ box, const int32_t* __restrict__ lmax,
                                          int32_t fb, const __grid_constant__ MmaArgs a, int4* __restrict__ frames) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntiles;
       t += (long long)gridDim.x * blockDim.x) {
    const int4 k = tblk[t];
    int4 bx = box[k.x];
    int lm = lmax[k.x];
    for (int h = 0; h < 2; ++h) {
      const int j = h ? k.z : k.y;
      if (j < 0) continue;
      const int4 q = box[j];
      bx = make_int4(min(bx.x, q.x), min(bx.y, q.y), max(bx.z, q.z), max(bx.w, q.w));
      lm = max(lm, lmax[j]);
    }
    const int ext = max(bx.z - bx.x, bx.w - bx.y);
    int b = ext > kMmaCoordMax ? (32 - __clz(ext)) - 10 : 0;
    while (b + fb < 30 && mma_radius(lm, fb, b + fb, a.cm[b + fb]) > kMmaCoordMax) ++b;
    frames[t] = make_int4(bx.x, bx.y, b, b + fb);
  }
}

constexpr size_t kMmaStage = (size_t)(kMmaI + kMmaJ) * 32;  // operand stage: i-rows | j-rows, 16 fp16 each
constexpr size_t kMmaPtStage = (size_t)(kMmaI + kMmaJ) * 16;  // point stage: i-points | j-points
constexpr size_t kMmaSmem = 120 * 1024;  // the stages, padded so that a CTA has the SM (and its 512 TMEM columns)
constexpr int kMmaPtStages = 5;  // point stages: copies run 3 tile pairs ahead, the epilogue reads the last one
constexpr int kMmaPtAhead = 3;
constexpr int kMmaSlice = 64;    // tile entries and frames copied 64 at a time, one slice ahead
static_assert(kMmaAcc * kMmaStage + kMmaPtStages * kMmaPtStage <= kMmaSmem, "stages");
static_assert((kMmaPtAhead + 1) % kMmaPtStages != 0 && kMmaPtAhead < kMmaSlice, "pipeline depths");

__device__ __forceinline__ void mma_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// bulk copy global -> shared, completion counted on the mbarrier (both addresses
// 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void mma_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}


// exact decision for a candidate of the tensor-core scan: positions ii < jj,
// their points {x, y, lambda, node}
__device__ __noinline__ void pricing_confirm4(const int4 pu, const int4 pv, int32_t fb,
                                              const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                              int2* pairs, long long cap, unsigned long long* count) {
  const long long S = (long long)pu.z + pv.z;
  if (S <= 0) return;
  const long long c = exact_cost(pu.x - pv.x, pu.y - pv.y);
  if ((c << fb) - S >= 0) return;
  const int i = min(pu.w, pv.w), j = max(pu.w, pv.w);
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

// the fp32 filter of the CUDA-core scan (pricing_filter, its radius s as in
// pricing_prep_kernel) on two points {x, y, lambda, node}: no false negatives
__device__ __forceinline__ bool mma_fp32_pass(const int4 pu, const int4 pv, int32_t fb) {
  const float scale = ldexpf(1.0f, -fb), grow = 1.0f + ldexpf(1.0f, -17);
  const float su = (fmaxf((float)pu.z * scale + 0.25f, 0.0f) + 2.0f) * grow;
  const float sv = (fmaxf((float)pv.z * scale + 0.25f, 0.0f) + 2.0f) * grow;
  const float xu = (float)pu.x, xv = (float)pv.x;
  return pricing_filter(xv - sv, xv + sv, (float)pv.y, -(xu - su), -(xu + su), -(float)pu.y) < 0.0f;
}

// lop3 0xFE: a | b | c
__device__ __forceinline__ uint32_t or3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0xFE;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__global__ void __launch_bounds__(kMmaThreads, 1) pricing_mma_kernel(const __grid_constant__ MmaArgs a) {
  // dynamic: operand stages [kMmaAcc][kMmaStage] | point stages [kMmaPtStages][kMmaPtStage]
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_pts_full[kMmaPtStages], s_pts_free[kMmaPtStages];
  __shared__ __align__(8) unsigned long long s_op_full[kMmaAcc], s_op_free[kMmaAcc], s_acc_full[kMmaAcc],
      s_acc_free[kMmaAcc], s_ent[2];
  __shared__ __align__(16) int4 s_tile[2][kMmaSlice];  // tile entries of slice k in buffer k mod 2
  __shared__ __align__(16) int4 s_frm[2][kMmaSlice];   // and their frames
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int fb = a.fb;
  // this CTA's tile pairs: a contiguous part of the list (iteration k takes t0 + k)
  const long long t0 = (long long)blockIdx.x * a.ntiles / gridDim.x;
  const int cnt = (int)((long long)(blockIdx.x + 1) * a.ntiles / gridDim.x - t0);
  uint8_t* const ostage = smem;
  const int4* const pstage = reinterpret_cast<const int4*>(smem + kMmaAcc * kMmaStage);
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  for (int r = tid; r < kMmaAcc * (kMmaI + kMmaJ); r += kMmaThreads) {  // K columns 8..15 stay zero
    const int stg = r / (kMmaI + kMmaJ), rr = r % (kMmaI + kMmaJ);
    uint8_t* base = ostage + stg * kMmaStage + (rr < kMmaI ? 0 : kMmaI * 32);
    *reinterpret_cast<uint4*>(base + tc::kmajor_off(rr < kMmaI ? rr : rr - kMmaI, 8, 16)) = zero;
  }
  auto u32 = [](const void* p) { return tc::smem_u32(p); };
  auto arrive = [&](unsigned long long* mb) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(u32(mb)) : "memory");
  };
  auto wait = [&](unsigned long long* mb, uint32_t parity) {
    const bool ok = tc::mbar_wait_sleep(u32(mb), parity, 4096, 1000000u);  // 4 s at most
    if (!ok) atomicOr(a.status, 1);
    return ok;
  };
  // slice k of the entries and frames (iterations 64k ..) into buffer k mod 2
  auto issue_slice = [&](int k) {
    const int first = k * kMmaSlice;
    if (first >= cnt) return;
    const uint32_t nb = (uint32_t)min(kMmaSlice, cnt - first) * 16u;
    mma_expect_tx(u32(&s_ent[k & 1]), 2u * nb);
    mma_bulk_g2s(u32(&s_tile[k & 1][0]), a.tiles + t0 + first, nb, u32(&s_ent[k & 1]));
    mma_bulk_g2s(u32(&s_frm[k & 1][0]), a.frames + t0 + first, nb, u32(&s_ent[k & 1]));
  };
  auto wait_entry = [&](int k) { return wait(&s_ent[(k / kMmaSlice) & 1], (uint32_t)((k / kMmaSlice / 2) & 1)); };
  auto entry = [&](int k) { return s_tile[(k / kMmaSlice) & 1][k % kMmaSlice]; };
  auto frame = [&](int k) { return s_frm[(k / kMmaSlice) & 1][k % kMmaSlice]; };

  if (warp == kMmaWarpMma) tc::tmem_alloc(u32(&s_tmem), kMmaAcc * kMmaJ);
  if (tid == 0) {
    for (int k = 0; k < kMmaPtStages; ++k) {
      tc::mbar_init(u32(&s_pts_full[k]), 1);
      tc::mbar_init(u32(&s_pts_free[k]), kMmaBuildWarps);
    }
    for (int k = 0; k < kMmaAcc; ++k) {
      tc::mbar_init(u32(&s_op_full[k]), kMmaBuildWarps);
      tc::mbar_init(u32(&s_op_free[k]), 1);
      tc::mbar_init(u32(&s_acc_full[k]), 1);
      tc::mbar_init(u32(&s_acc_free[k]), kMmaEpiWarps);
    }
    for (int k = 0; k < 2; ++k) tc::mbar_init(u32(&s_ent[k]), 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue_slice(0);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tacc = s_tmem;

  if (warp == kMmaWarpCopy) {
    // copies: the next slice of entries 16 tile pairs into a slice (the
    // epilogue, at most kMmaPtStages + kMmaAcc tile pairs behind, is done with
    // the buffer by then), each tile pair's points once its point stage is free
    if (lane == 0) {
      for (int k = 0; k < cnt; ++k) {
        if (k % kMmaSlice == 16) issue_slice(k / kMmaSlice + 1);
        if (!wait_entry(k)) break;
        const int st = k % kMmaPtStages;
        if (!wait(&s_pts_free[st], (uint32_t)(((k / kMmaPtStages) & 1) ^ 1))) break;
        const int4 l = entry(k);
        const uint32_t dst = u32(pstage + st * (kMmaI + kMmaJ));
        const uint32_t bi = (uint32_t)(l.y - l.x) * 16u, bj = (uint32_t)(l.w - l.z) * 16u;
        mma_expect_tx(u32(&s_pts_full[st]), bi + bj);
        mma_bulk_g2s(dst, a.pts4 + l.x, bi, u32(&s_pts_full[st]));
        mma_bulk_g2s(dst + kMmaI * 16, a.pts4 + l.z, bj, u32(&s_pts_full[st]));
      }
    }
  } else if (warp == kMmaWarpMma) {
    // tensor core: tile pair k once its operands are written and its accumulator is free
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f16(kMmaI, kMmaJ);
      for (int k = 0; k < cnt; ++k) {
        const int s2 = k % kMmaAcc;
        const uint32_t ph = (uint32_t)((k / kMmaAcc) & 1);
        if (!wait(&s_op_full[s2], ph)) break;
        if (!wait(&s_acc_free[s2], ph ^ 1u)) break;
        tc::fence_after();
        uint8_t* sA = ostage + s2 * kMmaStage;
        const uint64_t adesc = tc::smem_desc(u32(sA), 16);
        const uint64_t bdesc = tc::smem_desc(u32(sA + kMmaI * 32), 16);
        tc::mma_bf16(tacc + (uint32_t)(s2 * kMmaJ), adesc, bdesc, idesc, 0u);
        tc::commit(u32(&s_acc_full[s2]));
        tc::commit(u32(&s_op_free[s2]));
      }
    }
    __syncwarp();
  } else if (warp >= kMmaWarpBuild && warp < kMmaWarpBuild + kMmaBuildWarps) {
    // operand rows: i-row bt (bt < 128) or j-row bt - 128 of every tile pair
    const int bt = tid - kMmaWarpBuild * 32;
    const bool irow = bt < kMmaI;
    const int row = irow ? bt : bt - kMmaI;
    for (int k = 0; k < cnt; ++k) {
      const int s2 = k % kMmaAcc, st = k % kMmaPtStages;
      const bool ok = wait_entry(k) && wait(&s_pts_full[st], (uint32_t)((k / kMmaPtStages) & 1)) &&
                      wait(&s_op_free[s2], (uint32_t)(((k / kMmaAcc) & 1) ^ 1));
      const int4 l = entry(k), fr = frame(k);
      const bool has = ok && (irow ? l.x + row < l.y : l.z + row < l.w);
      uint4 w = irow ? make_uint4(mma_pack_h2(1024, 0), mma_pack_h2(2048, 1), 0u, 0u)
                     : make_uint4(mma_pack_h2(2048, 1), mma_pack_h2(1024, 0), 0u, 0u);
      if (has) {
        const int4 pt = pstage[st * (kMmaI + kMmaJ) + bt];
        const int b = fr.z, m = fr.w;
        const int X = (pt.x - fr.x) >> b, Y = (pt.y - fr.y) >> b, R = mma_radius(pt.z, fb, m, a.cm[m]);
        const int A = X * X + Y * Y - R * R;
        w = irow ? make_uint4(mma_pack_h2(A >> 11, A & 2047), mma_pack_h2(2048, 1), mma_pack_h2(X, Y),
                              mma_pack_h2(R, 0))
                 : make_uint4(mma_pack_h2(2048, 1), mma_pack_h2(A >> 11, A & 2047), mma_pack_h2(-2 * X, -2 * Y),
                              mma_pack_h2(-2 * R, 0));
      }
      *reinterpret_cast<uint4*>(ostage + s2 * kMmaStage + (irow ? 0 : kMmaI * 32) + tc::kmajor_off(row, 0, 16)) = w;
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        arrive(&s_op_full[s2]);
        arrive(&s_pts_free[st]);  // the points are no longer needed
      }
    }
  } else if (warp >= kMmaWarpEpi) {
    // accumulators: warp w reads lanes 32 (w mod 4) .. + 31 and 32 columns; a
    // negative value is appended to the candidate list (decided by the next kernel)
    const int q = warp & 3, cb = (warp - kMmaWarpEpi) >> 2;
    for (int k = 0; k < cnt; ++k) {
      const int s2 = k % kMmaAcc;
      const bool okm = wait(&s_acc_full[s2], (uint32_t)((k / kMmaAcc) & 1)) && wait_entry(k);
      tc::fence_after();
      const int4 tl = entry(k);
      const uint32_t taddr = tacc + (uint32_t)(s2 * kMmaJ) + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cb);
      uint32_t v[32];
      tc::tmem_ld32_issue(taddr, v);
      tc::tmem_wait_ld();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) arrive(&s_acc_free[s2]);  // the accumulator is free once read
      uint32_t o = or3(v[0], v[1], v[2]);
#pragma unroll
      for (int kk = 3; kk + 1 < 32; kk += 2) o = or3(o, v[kk], v[kk + 1]);
      o |= v[31];
      const int ii = tl.x + 32 * q + lane;
      const bool neg = okm && (int)o < 0 && ii < tl.y;
      if (__ballot_sync(0xffffffffu, neg)) {  // rare: append the negative ones
        uint32_t nm = 0u;
        if (neg) {
#pragma unroll
          for (int kk = 0; kk < 32; ++kk) nm |= (v[kk] >> 31) << kk;
          const int j0 = tl.z + 32 * cb;
          // only pairs ii < jj inside the tile pair
          const int lo = ii + 1 - j0, hi = tl.w - j0;  // columns [lo, hi)
          const uint32_t below = lo <= 0 ? 0u : (lo >= 32 ? 0xffffffffu : ((1u << lo) - 1u));
          const uint32_t above = hi >= 32 ? 0u : (hi <= 0 ? 0xffffffffu : ~((1u << hi) - 1u));
          nm &= ~(below | above);
        }
        const int c_n = __popc(nm);
        int incl = c_n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 31 && total) base = atomicAdd(a.ncand, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 31);
        unsigned long long at = base + (unsigned long long)(incl - c_n);
        const int j0 = tl.z + 32 * cb;
        while (nm) {
          const int kk = __ffs(nm) - 1;
          nm &= nm - 1u;
          if ((long long)at < a.cand_cap) a.cand[at] = make_int2(ii, j0 + kk);
          ++at;
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == kMmaWarpMma) tc::tmem_dealloc(tacc, kMmaAcc * kMmaJ);
}

// the candidates of a scan, decided: the fp32 filter, then exactly
__global__ void pricing_mma_confirm_kernel(const __grid_constant__ MmaArgs a) {
  const unsigned long long nc = *a.ncand;
  const long long n = (long long)nc < a.cand_cap ? (long long)nc : a.cand_cap;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int2 c = a.cand[t];
    const int4 pu = a.pts4[c.x], pv = a.pts4[c.y];
    if (mma_fp32_pass(pu, pv, a.fb)) pricing_confirm4(pu, pv, a.fb, a.rp, a.ec, a.pairs, a.cap, a.count);
  }
}

// C_m = ceil(sqrt(2^(2m+3))) for m = 0 .. 30, by exact integer arithmetic
static void mma_cm_table(long long* cm, int count) {
  for (int m = 0; m < count; ++m) {
    if (m > 30) {
      cm[m] = cm[30];  // never used: every radius fits by m = 30 (|lambda| < 2^29)
      continue;
    }
    const unsigned __int128 t = (unsigned __int128)1 << (2 * m + 3);
    unsigned long long k = (unsigned long long)std::sqrt((long double)t);
    while ((unsigned __int128)k * k > t) --k;
    while ((unsigned __int128)(k + 1) * (k + 1) <= t) ++k;
    cm[m] = (long long)((unsigned __int128)k * k == t ? k : k + 1);
  }
}

cudaError_t launch_pricing_mma_prep(const int2* xy, const int32_t* lam, const int32_t* perm, int32_t n,
                                    int4* pts4, cudaStream_t st) {
  const int threads = 256;
  int blocks = (int)((n + threads - 1) / threads);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  pricing_mma_prep_kernel<<<blocks, threads, 0, st>>>(xy, lam, perm, n, pts4);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pricing_mma_scan(const int4* pts4, const int2* xy, const int32_t* lam, const int32_t* rp,
                                    const int2* ec, int32_t fb, const int4* tiles, const int4* tblk,
                                    int32_t ntiles, const int2* ranges, int32_t nblocks, int4* box, int32_t* lmax,
                                    int4* frames, int2* cand, int64_t cand_cap, unsigned long long* ncand,
                                    int2* pairs, int64_t cap, unsigned long long* count,
                                    unsigned int* tile_counter, int32_t* status, int num_sms, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(ncand, 0, sizeof(unsigned long long), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(tile_counter, 0, sizeof(unsigned int), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  if (err != cudaSuccess) return err;
  if (ntiles == 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    err = cudaFuncSetAttribute(pricing_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmaSmem);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  MmaArgs a;
  a.pts4 = pts4;
  a.tiles = tiles;
  a.frames = frames;
  a.ntiles = ntiles;
  a.fb = fb;
  a.xy = xy;
  a.lam = lam;
  a.rp = rp;
  a.ec = ec;
  a.pairs = pairs;
  a.cap = cap;
  a.count = count;
  a.tile_counter = tile_counter;
  a.status = status;
  a.cand = cand;
  a.ncand = ncand;
  a.cand_cap = cand_cap;
  mma_cm_table(a.cm, 40);
  pricing_mma_blocks_kernel<<<(int)(((long long)nblocks * 32 + 255) / 256), 256, 0, st>>>(pts4, ranges, nblocks,
                                                                                          box, lmax);
  count_launch();
  int fgrid = (int)((ntiles + 255) / 256);
  if (fgrid > 4096) fgrid = 4096;
  pricing_mma_frames_kernel<<<fgrid, 256, 0, st>>>(tblk, ntiles, box, lmax, fb, a, frames);
  count_launch();
  int grid = num_sms;
  if (grid > ntiles) grid = ntiles;
  pricing_mma_kernel<<<grid, kMmaThreads, kMmaSmem, st>>>(a);
  count_launch();
  pricing_mma_confirm_kernel<<<num_sms * 4, 256, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

// ---- Check of the tensor-core arithmetic the scan relies on ----------------------
//
// One CTA, `rounds` times: operand rows drawn at random within the ranges the
// scan produces (A_hi in [-512, 1023] or the 1024 of a padding row, A_lo in
// [0, 2047], X, Y, R in [0, 1023], values at the ends of the ranges half of
// the time), one 128 x 256 x 16 MMA as in the scan, and every accumulator value
// compared with the exact integer product (int64 on the CUDA cores).

__device__ __forceinline__ uint32_t mma_check_hash(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return (uint32_t)(x ^ (x >> 31));
}

// a value in [lo, hi]: an end of the range half of the time
__device__ __forceinline__ int mma_check_draw(unsigned long long key, int lo, int hi) {
  const uint32_t h = mma_check_hash(key);
  if (h & 1u) return (h & 2u) ? hi : lo;
  return lo + (int)((h >> 2) % (uint32_t)(hi - lo + 1));
}

__global__ void __launch_bounds__(kMmaI, 1) pricing_mma_check_kernel(long long rounds, unsigned long long seed,
                                                                     unsigned long long* checked,
                                                                     unsigned long long* mismatches,
                                                                     int32_t* status) {
  __shared__ __align__(128) uint8_t sA[kMmaI * 32];
  __shared__ __align__(128) uint8_t sB[kMmaJ * 32];
  __shared__ short sBv[kMmaJ][8];  // the j-rows' first 8 entries, as integers
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_mbar;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  *reinterpret_cast<uint4*>(sA + tc::kmajor_off(tid, 8, 16)) = zero;
  for (int h = 0; h < kMmaJ / kMmaI; ++h) *reinterpret_cast<uint4*>(sB + tc::kmajor_off(tid + h * kMmaI, 8, 16)) = zero;
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&s_tmem), kMmaJ);
  if (tid == 0) tc::mbar_init(tc::smem_u32(&s_mbar), 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tacc = s_tmem;
  constexpr uint32_t idesc = tc::idesc_f16(kMmaI, kMmaJ);
  const uint64_t adesc = tc::smem_desc(tc::smem_u32(sA), 16), bdesc = tc::smem_desc(tc::smem_u32(sB), 16);
  unsigned long long bad = 0, done = 0;
  uint32_t phase = 0;
  for (long long r = 0; r < rounds; ++r) {
    const unsigned long long base = (seed * 0x100000001B3ull + (unsigned long long)r) << 12;
    int av[8];
    {  // i-row: [A_hi, A_lo, 2048, 1, X, Y, R, 0], a padding row one time in 16
      const unsigned long long k = base + (unsigned long long)tid * 8;
      const bool pad = (mma_check_hash(k + 7) & 15u) == 0u;
      av[0] = pad ? 1024 : mma_check_draw(k, -512, 1023);
      av[1] = pad ? 0 : mma_check_draw(k + 1, 0, 2047);
      av[2] = 2048;
      av[3] = 1;
      av[4] = pad ? 0 : mma_check_draw(k + 2, 0, kMmaCoordMax);
      av[5] = pad ? 0 : mma_check_draw(k + 3, 0, kMmaCoordMax);
      av[6] = pad ? 0 : mma_check_draw(k + 4, 0, kMmaCoordMax);
      av[7] = 0;
      *reinterpret_cast<uint4*>(sA + tc::kmajor_off(tid, 0, 16)) =
          make_uint4(mma_pack_h2(av[0], av[1]), mma_pack_h2(av[2], av[3]), mma_pack_h2(av[4], av[5]),
                     mma_pack_h2(av[6], av[7]));
    }
    for (int h = 0; h < kMmaJ / kMmaI; ++h) {  // j-rows: [2048, 1, A_hi, A_lo, -2X, -2Y, -2R, 0]
      const int row = tid + h * kMmaI;
      const unsigned long long k = base + 4096 + (unsigned long long)row * 8;
      const bool pad = (mma_check_hash(k + 7) & 15u) == 0u;
      int bv[8];
      bv[0] = 2048;
      bv[1] = 1;
      bv[2] = pad ? 1024 : mma_check_draw(k, -512, 1023);
      bv[3] = pad ? 0 : mma_check_draw(k + 1, 0, 2047);
      bv[4] = pad ? 0 : -2 * mma_check_draw(k + 2, 0, kMmaCoordMax);
      bv[5] = pad ? 0 : -2 * mma_check_draw(k + 3, 0, kMmaCoordMax);
      bv[6] = pad ? 0 : -2 * mma_check_draw(k + 4, 0, kMmaCoordMax);
      bv[7] = 0;
      for (int q = 0; q < 8; ++q) sBv[row][q] = (short)bv[q];
      *reinterpret_cast<uint4*>(sB + tc::kmajor_off(row, 0, 16)) =
          make_uint4(mma_pack_h2(bv[0], bv[1]), mma_pack_h2(bv[2], bv[3]), mma_pack_h2(bv[4], bv[5]),
                     mma_pack_h2(bv[6], bv[7]));
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      tc::mma_bf16(tacc, adesc, bdesc, idesc, 0u);
      tc::commit(tc::smem_u32(&s_mbar));
    }
    const bool ok = tc::mbar_wait(tc::smem_u32(&s_mbar), phase, kMmaWaitLimit);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(status, 1);
      break;
    }
    tc::fence_after();
    const uint32_t trow = tacc + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < kMmaJ; c0 += 32) {
      float v[32];
      tc::tmem_ld32(trow + (uint32_t)c0, v);
      for (int k = 0; k < 32; ++k) {
        long long e = 0;
        for (int q = 0; q < 8; ++q) e += (long long)av[q] * sBv[c0 + k][q];
        bad += ((long long)v[k] != e || v[k] != (float)e) ? 1ull : 0ull;
        ++done;
      }
    }
    tc::fence_before();
    __syncthreads();  // the rows are rewritten next round
  }
  atomicAdd(checked, done);
  atomicAdd(mismatches, bad);
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tacc, kMmaJ);
}

cudaError_t launch_pricing_mma_check(long long rounds, unsigned long long seed, unsigned long long* checked,
                                     unsigned long long* mismatches, int32_t* status, cudaStream_t st) {
  pricing_mma_check_kernel<<<1, kMmaI, 0, st>>>(rounds, seed, checked, mismatches, status);
  count_launch();
  return cudaGetLastError();
}
}  // namespace f2m
