// Per-row order statistics for the GDP kernels (gdp.cu): the two adjusted
// values a node's update needs (Eq. 10 for b_v = 2; Section 3 with Eq. 8, the
// b_v-th and (b_v+1)-th, in general), computed by a group of G lanes that
// stream the row.  Each also adds min(0, z) of the lane's entries to b2.
#pragma once

#include <climits>

#include "f2m_device.cuh"

namespace f2m {

// z(2) and z(3) of the row: lane-private top-3, merged over the group with xor
// shuffles
template <int G>
__device__ __forceinline__ void row_order_pair_f2m(const int2* __restrict__ ec, const int32_t* lin,
                                                   int beg, int end, int sub, unsigned gmask,
                                                   int lv, int F, long long& b2, int& z1, int& z2) {
  int a = INT_MAX, b = INT_MAX, c = INT_MAX;
#pragma unroll 4
  for (int e = beg + sub; e < end; e += G) {
    const int2 q = __ldg(ec + e);
    const int z = (q.y << F) - lv - ld_cg(lin + q.x);  // Eq. 9
    b2 += min(z, 0);
    top3_insert(z, a, b, c);
  }
  if (G > 1) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const int pa = __shfl_xor_sync(gmask, a, o);
      const int pb = __shfl_xor_sync(gmask, b, o);
      const int pc = __shfl_xor_sync(gmask, c, o);
      top3_insert(pa, a, b, c);
      top3_insert(pb, a, b, c);
      top3_insert(pc, a, b, c);
    }
  }
  z1 = b;
  z2 = c;
}

constexpr int kTopK = 8;

// keep the K smallest values seen, ascending, in registers
template <int K>
__device__ __forceinline__ void topk_insert(int z, int (&a)[K]) {
  if (z < a[K - 1]) {
    a[K - 1] = z;
#pragma unroll
    for (int k = K - 1; k > 0; --k) {
      const int lo = min(a[k - 1], a[k]), hi = max(a[k - 1], a[k]);
      a[k - 1] = lo;
      a[k] = hi;
    }
  }
}

// the K smallest of two ascending lists, ascending: min(a[k], p[K-1-k]) is a
// bitonic sequence holding them, which a bitonic merge sorts
template <int K>
__device__ __forceinline__ void topk_merge(int (&a)[K], const int (&p)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = min(a[k], p[K - 1 - k]);
#pragma unroll
  for (int s = K / 2; s > 0; s >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if ((k & s) == 0) {
        const int lo = min(a[k], a[k + s]), hi = max(a[k], a[k + s]);
        a[k] = lo;
        a[k + s] = hi;
      }
    }
  }
}

// z(bv) and z(bv+1) of row v (1-based order statistics of the adjusted values),
// also adding min(0, z) of the lane's entries to b2.  Every lane of the group
// returns the same pair.  Registers: needs bv + 1 <= kTopK.
template <int G>
__device__ __forceinline__ void row_order_pair_topk(const int2* __restrict__ ec, const int32_t* lin,
                                                    int beg, int end, int sub, unsigned gmask,
                                                    int lv, int F, int bv, long long& b2, int& z1,
                                                    int& z2) {
  int a[kTopK];
#pragma unroll
  for (int k = 0; k < kTopK; ++k) a[k] = INT_MAX;
  for (int e = beg + sub; e < end; e += G) {
    const int2 q = __ldg(ec + e);
    const int z = (q.y << F) - lv - ld_cg(lin + q.x);  // Eq. 9
    b2 += min(z, 0);
    topk_insert(z, a);
  }
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    int p[kTopK];
#pragma unroll
    for (int k = 0; k < kTopK; ++k) p[k] = __shfl_xor_sync(gmask, a[k], o);
    topk_merge(a, p);
  }
  z1 = INT_MAX;
  z2 = INT_MAX;
#pragma unroll
  for (int k = 0; k < kTopK; ++k) {
    if (k == bv - 1) z1 = a[k];
    if (k == bv) z2 = a[k];
  }
}

// the same by counting, for any bv: the entry value t is z(r) iff
// #{z < t} < r <= #{z <= t}; each lane tests its own entries against the row
template <int G>
__device__ __forceinline__ void row_order_pair_count(const int2* __restrict__ ec, const int32_t* lin,
                                                     int beg, int end, int sub, unsigned gmask,
                                                     int lv, int F, int bv, long long& b2, int& z1,
                                                     int& z2) {
  int c1 = INT_MAX, c2 = INT_MAX;
  for (int j = beg + sub; j < end; j += G) {
    const int2 qj = __ldg(ec + j);
    const int zj = (qj.y << F) - lv - ld_cg(lin + qj.x);  // Eq. 9
    b2 += min(zj, 0);
    int lt = 0, le = 0;
    for (int e = beg; e < end; ++e) {
      const int2 q = __ldg(ec + e);
      const int z = (q.y << F) - lv - ld_cg(lin + q.x);
      lt += (z < zj);
      le += (z <= zj);
    }
    if (lt < bv && bv <= le) c1 = min(c1, zj);
    if (lt <= bv && bv + 1 <= le) c2 = min(c2, zj);
  }
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    c1 = min(c1, __shfl_xor_sync(gmask, c1, o));
    c2 = min(c2, __shfl_xor_sync(gmask, c2, o));
  }
  z1 = c1;
  z2 = c2;
}

// b_v of node v and its pair of order statistics: MODE 0: b_v = 2 (Eq. 10,
// top-3); 1: b_v read from bdeg, all b_v < kTopK (registers); 2: b_v read from
// bdeg, any value (counting)
template <int G, int MODE>
__device__ __forceinline__ int row_order_pair(const int2* __restrict__ ec, const int32_t* lin,
                                              const int32_t* __restrict__ bdeg, long long v,
                                              int beg, int end, int sub, unsigned gmask, int lv,
                                              int F, long long& b2, int& z1, int& z2) {
  if constexpr (MODE == 1) {
    const int bv = __ldg(bdeg + v);
    row_order_pair_topk<G>(ec, lin, beg, end, sub, gmask, lv, F, bv, b2, z1, z2);
    return bv;
  } else if constexpr (MODE == 2) {
    const int bv = __ldg(bdeg + v);
    row_order_pair_count<G>(ec, lin, beg, end, sub, gmask, lv, F, bv, b2, z1, z2);
    return bv;
  } else {
    row_order_pair_f2m<G>(ec, lin, beg, end, sub, gmask, lv, F, b2, z1, z2);
    return 2;
  }
}

}  // namespace f2m
