// GDP phase, two sweeps per device-wide barrier (the default single-instance
// form when its tiles fit in shared memory).
//
// The sweep is the Jacobi step of Eq. 9 and Eq. 10 (Section 5.1), as in
// gdp_tiled.cu, and every result is bit-identical to it and to the oracle.
// What changes is how often the CTAs meet: each CTA also keeps the rows of its
// halo (H1: outside nodes adjacent to its own nodes) and the lambda of the
// second halo ring (H2: outside nodes adjacent to H1).  Per round it loads the
// lambda of H1 and H2 once, computes sweep 2r for its own rows and the H1 rows
// (the latter redundantly: their owners compute the same integers), then sweep
// 2r+1 for its own rows, whose neighbours are all own or H1 nodes, publishes
// its own lambda and meets the others at one barrier.  Integer arithmetic
// makes the redundant values identical, so nothing but the barrier count
// changes: one barrier and one halo load per two sweeps.
//
// The totals of round r (bound and changed count of both sweeps, overflow
// flags) are read by every CTA at the start of round r+1, overlapped with the
// halo load; the stop test then selects the buffer that holds the result.  An
// overflow in the second sweep of a round leaves the exact state (the input of
// that sweep) unmaterialised: the kernel reports it and the host replays the
// round with the one-sweep kernel, which stops at the same place.
#include <climits>
#include <type_traits>
#include <vector>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

namespace {

#define F2M_GRID_STRIDE2(i, count) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (count); \
       i += (long long)gridDim.x * blockDim.x)

constexpr int kSortCap2 = 16384;  // shared-memory sort capacity of the plan kernels

template <typename T>
cudaError_t grow2(T** p, int64_t* cap, int64_t need) {
  if (*p && *cap >= need) return cudaSuccess;
  if (*p) dev_free(*p);
  *p = nullptr;
  *cap = 0;
  const int64_t c = need + (need >> 3) + 64;
  cudaError_t e = dev_malloc((void**)p, sizeof(T) * (size_t)c);
  if (e == cudaSuccess) *cap = c;
  return e;
}

// ascending bitonic sort of s[0, m) in shared memory (padded with INT_MAX to a
// power of two P <= cap); returns P
__device__ int block_sort(int* s, int m) {
  const int tid = threadIdx.x, T = blockDim.x;
  int P = 1;
  while (P < m) P <<= 1;
  for (int i = m + tid; i < P; i += T) s[i] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += T) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int a = s[i], c = s[ixj];
          const bool up = (i & k) == 0;
          if ((a > c) == up) {
            s[i] = c;
            s[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  return P;
}

// degree-descending order of m nodes (ties by position): keys
// (2047 - min(deg, 2047)) << 20 | position, sorted ascending
__device__ void sort_by_degree(const int32_t* __restrict__ irp, const int32_t* nodes_or_null, int lo, int m,
                               int* s_key) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int g = nodes_or_null ? nodes_or_null[i] : lo + i;
    const int d = irp[g + 1] - irp[g];
    s_key[i] = ((2047 - min(d, 2047)) << 20) | i;
  }
  __syncthreads();
  block_sort(s_key, m);
}

__device__ __forceinline__ int lower_bound_g(const int32_t* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Pass 1: the second halo ring H2 of each CTA (sorted, into tmp2[b * cap]),
// and the sizes of the two-sweep tile.  H1 is the halo list of the one-sweep
// plan (tmp + irp[lo], hcount[b] entries, sorted).
// stats: [0] max sliced entries (own + H1 rows), [1] max slices, [2] max lambda
// slots (own + H1 + H2), [3] max halo (H1 + H2), [4] 1 if some CTA overflows
// the sort capacity
__global__ void plan_h2_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                               const int32_t* __restrict__ part, const int32_t* __restrict__ tmp,
                               const int32_t* __restrict__ hcount, const int32_t* __restrict__ scount,
                               int32_t* __restrict__ tmp2, int32_t* __restrict__ h2count,
                               int32_t* __restrict__ hhcount, int32_t* __restrict__ s2count,
                               int32_t* __restrict__ nslc, int32_t* __restrict__ stats) {
  extern __shared__ int s_sort[];
  __shared__ int s_cnt;
  __shared__ int s_warp[33];
  const int b = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int H1 = hcount[b];
  const int32_t* h1 = tmp + irp[lo];
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int i = tid; i < H1; i += T) {
    const int h = h1[i];
    for (int e = irp[h]; e < irp[h + 1]; ++e) {
      const int c = iec[e].x;
      if (c >= lo && c < hi) continue;
      const int p = lower_bound_g(h1, H1, c);
      if (p < H1 && h1[p] == c) continue;
      const int k = atomicAdd(&s_cnt, 1);
      if (k < kSortCap2) s_sort[k] = c;
    }
  }
  __syncthreads();
  const int m = s_cnt;
  if (m > kSortCap2 || H1 > kSortCap2 || own > kSortCap2) {
    if (tid == 0) {
      atomicOr(&stats[4], 1);
      h2count[b] = 0;
      hhcount[b] = 0;
      s2count[b] = 0;
      nslc[b] = 0;
    }
    return;
  }
  block_sort(s_sort, m);
  // distinct values in order into tmp2
  const int chunk = (m + T - 1) / T;
  const int i0 = min(m, tid * chunk), i1 = min(m, i0 + chunk);
  int cnt = 0;
  for (int i = i0; i < i1; ++i) cnt += (i == 0 || s_sort[i] != s_sort[i - 1]);
  int H2 = 0;
  int o = block_exclusive_scan(cnt, s_warp, H2);
  for (int i = i0; i < i1; ++i)
    if (i == 0 || s_sort[i] != s_sort[i - 1]) tmp2[(size_t)b * kSortCap2 + o++] = s_sort[i];
  __syncthreads();
  // sliced size of the H1 rows
  sort_by_degree(irp, h1, 0, H1, s_sort);
  int sz = 0;
  for (int s = tid; s * 32 < H1; s += T) {
    const int g = h1[s_sort[s * 32] & 0xFFFFF];
    sz += 32 * (irp[g + 1] - irp[g]);
  }
  int s1 = 0;
  block_exclusive_scan(sz, s_warp, s1);
  if (tid == 0) {
    const int slices = (own + 31) / 32 + (H1 + 31) / 32;
    h2count[b] = H2;
    hhcount[b] = H1 + H2;
    s2count[b] = scount[b] + s1;
    nslc[b] = slices;
    atomicMax(&stats[0], scount[b] + s1);
    atomicMax(&stats[1], slices);
    atomicMax(&stats[2], own + H1 + H2);
    atomicMax(&stats[3], H1 + H2);
  }
}

// Pass 2: halo lists (H1 then H2), slot order, slice table and sliced entries.
//   slots 32 s + lane: own slices first (degree-descending own nodes), then
//   H1 slices; order2 = local node of a slot (own: 0..own-1, H1: own + i);
//   entries {local index, cost * 2^F}, local index own | own + H1 position |
//   own + H1 + H2 position; short rows padded with {zero slot, 2^30}.
__global__ void plan_map2_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                 const int32_t* __restrict__ part, const int32_t* __restrict__ tmp,
                                 const int32_t* __restrict__ hcount, const int32_t* __restrict__ tmp2,
                                 const int32_t* __restrict__ h2count, const int32_t* __restrict__ hoff2,
                                 const int32_t* __restrict__ soff2, const int32_t* __restrict__ sloff2,
                                 int32_t F, int32_t* __restrict__ halo2, int32_t* __restrict__ order2,
                                 int2* __restrict__ slc2, int2* __restrict__ lec2) {
  extern __shared__ int s_keys[];
  __shared__ int s_warp[33];
  const int b = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int H1 = hcount[b], H2 = h2count[b];
  const int32_t* h1 = tmp + irp[lo];
  const int32_t* h2 = tmp2 + (size_t)b * kSortCap2;
  const int zero_slot = own + H1 + H2;
  int* k_own = s_keys;               // [P(own)]
  int* k_h1 = s_keys + kSortCap2;    // [P(H1)]
  for (int i = tid; i < H1; i += T) halo2[hoff2[b] + i] = h1[i];
  for (int i = tid; i < H2; i += T) halo2[hoff2[b] + H1 + i] = h2[i];
  sort_by_degree(irp, nullptr, lo, own, k_own);
  sort_by_degree(irp, h1, 0, H1, k_h1);
  const int nslo = (own + 31) / 32, nsl1 = (H1 + 31) / 32, nsl = nslo + nsl1;
  // node (global internal id) of slot p, or -1 for a padding slot
  auto slot_node = [&](int p) -> int {
    if (p < 32 * nslo) return p < own ? lo + (k_own[p] & 0xFFFFF) : -1;
    const int q = p - 32 * nslo;
    return q < H1 ? h1[k_h1[q] & 0xFFFFF] : -1;
  };
  auto slot_local = [&](int p) -> int {
    if (p < 32 * nslo) return k_own[p] & 0xFFFFF;
    return own + (k_h1[p - 32 * nslo] & 0xFFFFF);
  };
  // slice offsets: exclusive scan of 32 * depth (depth = degree of the slice's first slot)
  const int chunk = (nsl + T - 1) / T;
  const int s0 = min(nsl, tid * chunk), s1 = min(nsl, s0 + chunk);
  int sz = 0;
  for (int s = s0; s < s1; ++s) {
    const int g = slot_node(32 * s);
    sz += 32 * (irp[g + 1] - irp[g]);
  }
  int total = 0;
  int base = block_exclusive_scan(sz, s_warp, total);
  const int sb = sloff2[b];
  for (int s = s0; s < s1; ++s) {
    const int g = slot_node(32 * s);
    const int depth = irp[g + 1] - irp[g];
    slc2[sb + s] = make_int2(base, depth);
    base += 32 * depth;
  }
  __syncthreads();
  int2* out = lec2 + soff2[b];
  for (int p = tid; p < nsl * 32; p += T) {
    const int s = p >> 5, lane = p & 31;
    const int2 sl = slc2[sb + s];
    const int g = slot_node(p);
    order2[(size_t)32 * sb + p] = g >= 0 ? slot_local(p) : zero_slot;
    const int a = g >= 0 ? irp[g] : 0, d = g >= 0 ? irp[g + 1] - irp[g] : 0;
    for (int k = 0; k < sl.y; ++k) {
      int2 q;
      if (k < d) {
        const int2 r = iec[a + k];
        int local;
        if (r.x >= lo && r.x < hi) {
          local = r.x - lo;
        } else {
          const int x = lower_bound_g(h1, H1, r.x);
          if (x < H1 && h1[x] == r.x) {
            local = own + x;
          } else {
            local = own + H1 + lower_bound_g(h2, H2, r.x);
          }
        }
        q = make_int2(local, r.y << F);  // cost in units 2^-F
      } else {
        q = make_int2(zero_slot, 1 << 30);
      }
      out[sl.x + k * 32 + lane] = q;
    }
  }
}

// one row of a slice: top-3 of z over the row (two chains) and, if BOUND, the
// row's bound term sum min(0, z)
// The sliced entries of one row (entry k of the row at index k * 32), as
// {local index, cost * 2^F}: stored as such (8 bytes), or packed into 4 bytes
// as cost << 13 | local index (cost below 2^19 - 1, local index below 2^13),
// which plan_build2 chooses when the 8-byte tiles do not fit shared memory.
struct EntWide {
  const int2* p;
  __device__ __forceinline__ int2 get(int k) const { return p[k * 32]; }
};
struct EntPacked {
  const uint32_t* p;
  int F;
  __device__ __forceinline__ int2 get(int k) const {
    const uint32_t e = p[k * 32];
    return make_int2((int)(e & 0x1FFFu), (int)(e >> 13) << F);
  }
};
template <bool PACKED>
__device__ __forceinline__ auto make_ent(const typename std::conditional<PACKED, uint32_t, int2>::type* p, int F) {
  if constexpr (PACKED) return EntPacked{p, F};
  else return EntWide{p};
}
constexpr uint32_t kPackPadCost = (1u << 19) - 1;  // cost of a packed padding entry
// lambda of the padding slot in the packed form: with cost kPackPadCost its z
// is about 2^30 - lambda_v, above every real one (as the 8-byte padding's)
constexpr int kPackPadLam = -(1 << 30) + (1 << 27);

template <bool BOUND, typename E>
__device__ __forceinline__ void row_top3(const E& ent, int depth, int lv, const int* s_in, int& bb, int& cc,
                                         long long& neg) {
  int a = INT_MAX, a1 = INT_MAX, b1 = INT_MAX, c1 = INT_MAX;
  bb = INT_MAX;
  cc = INT_MAX;
  neg = 0;
  int k = 0;
  for (; k + 1 < depth; k += 2) {
    const int2 q = ent.get(k), q1 = ent.get(k + 1);
    const int z = q.y - lv - s_in[q.x];  // Eq. 9
    const int z1 = q1.y - lv - s_in[q1.x];
    if (BOUND) neg += min(z, 0) + min(z1, 0);
    top3_insert_minmax(z, a, bb, cc);
    top3_insert_minmax(z1, a1, b1, c1);
  }
  if (k < depth) {
    const int2 q = ent.get(k);
    const int z = q.y - lv - s_in[q.x];
    if (BOUND) neg += min(z, 0);
    top3_insert_minmax(z, a, bb, cc);
  }
  top3_merge(a1, b1, c1, a, bb, cc);
}

// Degree requirements b_v (Section 3 with Eq. 8): z(b_v) and z(b_v + 1) of one
// row, and, if BOUND, the row's sum of min(0, z).  MODE 1 (every b_v < 8):
// the row's 8 smallest values kept sorted in registers; MODE 2: counting, the
// entry value t being z(r) iff #{z < t} < r <= #{z <= t}.  Slice padding
// entries have z above every real one and at least b_v + 1 entries are real.
template <bool BOUND, int MODE, typename E>
__device__ __forceinline__ void row_pair_deg(const E& ent, int depth, int lv, const int* s_in, int bv,
                                             int& z1, int& z2, long long& neg) {
  neg = 0;
  if constexpr (MODE == 1) {
    int a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = INT_MAX;
    for (int k = 0; k < depth; ++k) {
      const int2 q = ent.get(k);
      const int z = q.y - lv - s_in[q.x];  // Eq. 9
      if (BOUND) neg += min(z, 0);
      if (z < a[7]) {
        a[7] = z;
#pragma unroll
        for (int j = 7; j > 0; --j) {
          const int lo2 = min(a[j - 1], a[j]), hi2 = max(a[j - 1], a[j]);
          a[j - 1] = lo2;
          a[j] = hi2;
        }
      }
    }
    z1 = INT_MAX;
    z2 = INT_MAX;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k == bv - 1) z1 = a[k];
      if (k == bv) z2 = a[k];
    }
  } else {
    int c1 = INT_MAX, c2 = INT_MAX;
    for (int j = 0; j < depth; ++j) {
      const int2 qj = ent.get(j);
      const int zj = qj.y - lv - s_in[qj.x];  // Eq. 9
      if (BOUND) neg += min(zj, 0);
      int lt = 0, le = 0;
      for (int k = 0; k < depth; ++k) {
        const int2 q = ent.get(k);
        const int z = q.y - lv - s_in[q.x];
        lt += (z < zj);
        le += (z <= zj);
      }
      if (lt < bv && bv <= le) c1 = min(c1, zj);
      if (lt <= bv && bv + 1 <= le) c2 = min(c2, zj);
    }
    z1 = c1;
    z2 = c2;
  }
}

}  // namespace

// BOUND: also sum the dual bound of every sweep (only traces need it).
// MODE 0: b_v = 2 (Eq. 10, top-3); 1 and 2: b_v per node from bint (internal
// order), see row_pair_deg; these take 512 threads (more registers per row).
template <bool BOUND, int MODE, bool PACKED>
__global__ void __launch_bounds__(MODE == 0 ? 1024 : 512, 1)
gdp_tiled2_kernel(const int32_t* __restrict__ part, const int32_t* __restrict__ hcount,
                  const int32_t* __restrict__ hoff2, const int32_t* __restrict__ soff2,
                  const int32_t* __restrict__ sloff2, const int32_t* __restrict__ halo2,
                  const int32_t* __restrict__ order2, const int2* __restrict__ slc2,
                  const void* __restrict__ lec2v, int32_t* lam0, int32_t* lam1, int32_t shift,
                  long long max_sweeps, GdpCtl* ctl, long long* trace_b2, unsigned long long* trace_ch,
                  long long trace_cap, long long budget, int32_t maxS, int32_t maxSl, int32_t maxL,
                  int32_t maxHH, const int32_t* __restrict__ bint, int32_t F) {
  extern __shared__ __align__(16) unsigned char smem[];
  using EntT = typename std::conditional<PACKED, uint32_t, int2>::type;
  EntT* s_lec = reinterpret_cast<EntT*>(smem);         // sliced entries
  const int sS = PACKED ? ((maxS + 1) & ~1) : maxS;     // keeps what follows 8-byte aligned
  int2* s_slc = reinterpret_cast<int2*>(s_lec + sS);    // {offset, depth} per slice
  int* s_order = reinterpret_cast<int*>(s_slc + maxSl); // local node of each slot
  int* s_A = s_order + 32 * maxSl;                      // lambda: own | H1 | H2 | zero
  int* s_B = s_A + maxL + 1;
  int* s_hid = s_B + maxL + 1;                          // H1 then H2 node ids
  __shared__ long long s_b2[2][32];
  __shared__ unsigned s_ch[2][32];
  __shared__ int s_ovf[32];
  __shared__ int s_stop;

  const int tid = threadIdx.x, T = blockDim.x, b = blockIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int H1 = hcount[b];
  const int hb = hoff2[b], HH = hoff2[b + 1] - hb;
  const int S0 = soff2[b], S = soff2[b + 1] - S0;
  const int sb = sloff2[b], nsl = sloff2[b + 1] - sb;
  const int nslo = (own + 31) / 32;
  const int zero_slot = own + HH;
  const EntT* lec2 = reinterpret_cast<const EntT*>(lec2v);
  for (int e = tid; e < S; e += T) s_lec[e] = lec2[S0 + e];
  for (int s = tid; s < nsl; s += T) s_slc[s] = slc2[sb + s];
  for (int p = tid; p < 32 * nsl; p += T) s_order[p] = order2[(size_t)32 * sb + p];
  for (int h = tid; h < HH; h += T) s_hid[h] = halo2[hb + h];
  for (int i = tid; i < own; i += T) s_A[i] = lam0[lo + i];
  if (tid == 0) {
    s_A[zero_slot] = PACKED ? kPackPadLam : 0;
    s_B[zero_slot] = PACKED ? kPackPadLam : 0;
  }
  __syncthreads();
  volatile GdpCtl* vc = ctl;

  for (long long r = 0;; ++r) {
    const int32_t* lin = (r & 1) ? lam1 : lam0;
    int32_t* lout = (r & 1) ? lam0 : lam1;
    const long long t0 = 2 * r;
    // stop test on round r-1 (its totals are complete: every CTA added them
    // before arriving at barrier r-1), overlapped with this round's halo load
    if (tid == 0) {
      int stop = 0, res = (int)(r & 1);
      if (r >= 1) {
        const int ps = (int)((r - 1) % 3);
        const long long p0 = 2 * (r - 1), p1 = p0 + 1;
        const bool two = p1 < max_sweeps;
        const long long b0 = vc->slot_b2[ps], b1 = vc->q_b2[ps];
        const unsigned long long c0 = vc->slot_ch[ps], c1 = vc->q_ch[ps];
        const int of = vc->q_ovf[ps];
        long long done = -1;
        int st_bits = 0, fp = 0;
        const int in_buf = (int)((r - 1) & 1), out_buf = (int)(r & 1);
        // sweeps count the last sweep run (as the one-sweep kernel does)
        if (of & 1) {
          done = p0 + 1;
          st_bits = kGdpOverflow;
          res = in_buf;
        } else if (c0 == 0) {
          done = p0 + 1;
          fp = 1;
          res = in_buf;
        } else if (two && (of & 2)) {
          done = p1 + 1;
          st_bits = kGdpOddOverflow;
          res = in_buf;
        } else if (two && c1 == 0) {
          done = p1 + 1;
          fp = 1;
          res = out_buf;
        } else if (t0 >= max_sweeps) {
          done = max_sweeps;
          res = out_buf;
        }
        if (b == 0) {
          if (p0 < trace_cap) {
            trace_b2[p0] = b0;
            trace_ch[p0] = c0;
          }
          if (two && p1 < trace_cap && !(of & 1) && c0 != 0) {
            trace_b2[p1] = b1;
            trace_ch[p1] = c1;
          }
        }
        if (done >= 0) {
          stop = 1;
          if (b == 0) {
            vc->sweeps = done;
            vc->fixed_point = fp;
            vc->pad1 = res;
            if (st_bits) atomicOr(&ctl->status, st_bits);
          }
        }
      } else if (max_sweeps <= 0) {
        stop = 1;
        if (b == 0) {
          vc->sweeps = 0;
          vc->pad1 = 0;
        }
      }
      if (b == 0 && !stop) {  // slot (r+1)%3 was read during round r-1 and is next used in round r+1
        const int z = (int)((r + 1) % 3);
        vc->slot_b2[z] = 0;
        vc->slot_ch[z] = 0;
        vc->q_b2[z] = 0;
        vc->q_ch[z] = 0;
        vc->q_ovf[z] = 0;
      }
      s_stop = stop;
    }
    for (int h = tid; h < HH; h += T) s_A[own + h] = ld_cg(lin + s_hid[h]);
    __syncthreads();
    if (s_stop) break;

    // sweep t0: own rows and H1 rows, s_A -> s_B
    long long b2a = 0, b2b = 0;
    unsigned cha = 0, chb = 0;
    int ovfa = 0, ovfb = 0;
    for (int p = tid; p < 32 * nsl; p += T) {
      const int s = p >> 5;
      const bool is_own = s < nslo;
      if (is_own ? p >= own : (p - 32 * nslo) >= H1) continue;
      const int2 sl = s_slc[s];
      const int vl = s_order[p];
      const int lv = s_A[vl];
      int bb, cc, bv = 2;
      long long neg;
      const auto ent = make_ent<PACKED>(s_lec + sl.x + (p & 31), F);
      if constexpr (MODE == 0) {
        row_top3<BOUND>(ent, sl.y, lv, s_A, bb, cc, neg);
      } else {
        bv = __ldg(bint + (vl < own ? lo + vl : s_hid[vl - own]));
        row_pair_deg<BOUND, MODE>(ent, sl.y, lv, s_A, bv, bb, cc, neg);
      }
      const long long d = gdp_step(bb, cc, shift);  // Eq. 10 (Eq. 8), truncated toward 0
      const long long nl = (long long)lv + d;
      s_B[vl] = (int32_t)nl;
      if (is_own) {
        ovfa |= (nl >= kLamLimit || nl <= -kLamLimit);
        cha += (d != 0);
        if (BOUND) b2a += neg + 2LL * bv * lv;
      }
    }
    __syncthreads();
    const bool two = t0 + 1 < max_sweeps;
    if (two) {  // sweep t0 + 1: own rows, s_B -> s_A
      for (int p = tid; p < 32 * nslo; p += T) {
        if (p >= own) continue;
        const int2 sl = s_slc[p >> 5];
        const int vl = s_order[p];
        const int lv = s_B[vl];
        int bb, cc, bv = 2;
        long long neg;
        const auto ent = make_ent<PACKED>(s_lec + sl.x + (p & 31), F);
        if constexpr (MODE == 0) {
          row_top3<BOUND>(ent, sl.y, lv, s_B, bb, cc, neg);
        } else {
          bv = __ldg(bint + lo + vl);
          row_pair_deg<BOUND, MODE>(ent, sl.y, lv, s_B, bv, bb, cc, neg);
        }
        const long long d = gdp_step(bb, cc, shift);
        const long long nl = (long long)lv + d;
        s_A[vl] = (int32_t)nl;
        ovfb |= (nl >= kLamLimit || nl <= -kLamLimit);
        chb += (d != 0);
        if (BOUND) b2b += neg + 2LL * bv * lv;
      }
      __syncthreads();
    }
    const int* src = two ? s_A : s_B;
    for (int i = tid; i < own; i += T) lout[lo + i] = src[i];
    if (!two)
      for (int i = tid; i < own; i += T) s_A[i] = s_B[i];
    // totals of round r go in before this block arrives, so that they are
    // complete for everyone who has passed barrier r
    b2a = warp_sum_ll(b2a);
    b2b = warp_sum_ll(b2b);
    cha = warp_sum_u(cha);
    chb = warp_sum_u(chb);
    const int ovf = (__any_sync(0xffffffffu, ovfa) ? 1 : 0) | (__any_sync(0xffffffffu, ovfb) ? 2 : 0);
    if (lane == 0) {
      s_b2[0][warp] = b2a;
      s_b2[1][warp] = b2b;
      s_ch[0][warp] = cha;
      s_ch[1][warp] = chb;
      s_ovf[warp] = ovf;
    }
    __syncthreads();
    if (warp == 0) {
      long long x0 = lane < nwarps ? s_b2[0][lane] : 0, x1 = lane < nwarps ? s_b2[1][lane] : 0;
      unsigned y0 = lane < nwarps ? s_ch[0][lane] : 0, y1 = lane < nwarps ? s_ch[1][lane] : 0;
      int o = lane < nwarps ? s_ovf[lane] : 0;
      x0 = warp_sum_ll(x0);
      x1 = warp_sum_ll(x1);
      y0 = warp_sum_u(y0);
      y1 = warp_sum_u(y1);
      o = (int)__reduce_or_sync(0xffffffffu, (unsigned)o);
      if (lane == 0) {
        const int s = (int)(r % 3);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->slot_b2[s]), (unsigned long long)x0);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->q_b2[s]), (unsigned long long)x1);
        if (y0) atomicAdd(&ctl->slot_ch[s], (unsigned long long)y0);
        if (y1) atomicAdd(&ctl->q_ch[s], (unsigned long long)y1);
        if (o) atomicOr(&ctl->q_ovf[s], o);
        grid_arrive_counted(&ctl->bar_count);
        if (!grid_wait_counted(&ctl->bar_count, (unsigned)(r + 1) * gridDim.x, budget)) {
          atomicOr(&ctl->status, kGdpTimeout);
          s_stop = 1;
        } else {
          s_stop = 0;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
  }
}

// ---- host side -------------------------------------------------------------------------

void plan2_free(GdpPlan& p) {
  void* ptrs[] = {p.h2count, p.hhcount, p.s2count, p.nslc, p.hoff2, p.soff2, p.sloff2, p.halo2,
                  p.order2, p.slc2, p.lec2, p.tmp2, p.stats2, p.lec2p};
  for (void* q : ptrs)
    if (q) dev_free(q);
  p.h2count = p.hhcount = p.s2count = p.nslc = p.hoff2 = p.soff2 = p.sloff2 = p.halo2 = p.order2 = nullptr;
  p.tmp2 = p.stats2 = nullptr;
  p.slc2 = nullptr;
  p.lec2 = nullptr;
  p.lec2p = nullptr;
  p.lec2p_cap = 0;
  p.packed2 = false;
  p.cap2_small = p.halo2_cap = p.order2_cap = p.slc2_cap = p.lec2_cap = p.tmp2_cap = 0;
  p.valid2 = false;
}

#define P2CK(call)                              \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return e_;           \
  } while (0)

// 4-byte form of the sliced entries: cost << 13 | local index; the padding
// entries (cost field 1 << 30) become kPackPadCost.  *bad counts entries that
// do not pack (cost >= kPackPadCost or local index >= 2^13).
__global__ void plan_pack2_kernel(const int2* __restrict__ lec, int32_t m, int32_t F, uint32_t* __restrict__ out,
                                  int32_t* bad) {
  F2M_GRID_STRIDE2(i, m) {
    const int2 q = lec[i];
    const uint32_t c = q.y == (1 << 30) ? kPackPadCost : (uint32_t)(q.y >> F);
    if ((q.y != (1 << 30) && c >= kPackPadCost) || q.x < 0 || q.x >= (1 << 13)) atomicAdd(bad, 1);
    out[i] = (c << 13) | (uint32_t)(q.x & 0x1FFF);
  }
}

cudaError_t plan_build2(GdpPlan& p, int32_t F, cudaStream_t st) {
  p.valid2 = false;
  if (!p.valid || p.threads != 1024) return cudaSuccess;  // one CTA of 1024 threads per SM
  const int B = p.B;
  if (p.cap2_small < B + 1) {
    int64_t c = 0;
    for (int32_t** q : {&p.h2count, &p.hhcount, &p.s2count, &p.nslc, &p.hoff2, &p.soff2, &p.sloff2}) {
      if (*q) dev_free(*q);
      *q = nullptr;
      c = 0;
      P2CK(grow2(q, &c, B + 1));
    }
    p.cap2_small = B + 1;
  }
  if (!p.stats2) {
    int64_t c = 0;
    P2CK(grow2(&p.stats2, &c, 8));
  }
  P2CK(grow2(&p.tmp2, &p.tmp2_cap, (int64_t)B * kSortCap2));
  P2CK(cudaMemsetAsync(p.stats2, 0, 8 * sizeof(int32_t), st));
  const size_t sort_smem = kSortCap2 * sizeof(int32_t);
  P2CK(cudaFuncSetAttribute(plan_h2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem));
  plan_h2_kernel<<<B, 512, sort_smem, st>>>(p.irp, p.iec, p.part, p.tmp, p.hcount, p.scount, p.tmp2,
                                            p.h2count, p.hhcount, p.s2count, p.nslc, p.stats2);
  count_launch();
  P2CK(cudaGetLastError());
  int32_t stats[8];
  P2CK(cudaMemcpyAsync(stats, p.stats2, sizeof(stats), cudaMemcpyDeviceToHost, st));
  P2CK(cudaStreamSynchronize(st));
  if (stats[4]) return cudaSuccess;
  // shared memory per CTA: entries (8 bytes, or 4 packed), slices, slot
  // order, two lambda buffers, halo ids
  const int64_t rest = 8LL * stats[1] + 4LL * 32 * stats[1] + 8LL * (stats[2] + 1) + 4LL * stats[3];
  const int64_t smem8 = 8LL * stats[0] + rest;
  const int64_t smem4 = 4LL * ((stats[0] + 1) & ~1) + rest;
  int dev = 0, smem_optin = 0, smem_sm = 0;
  P2CK(cudaGetDevice(&dev));
  P2CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  P2CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  auto fits = [&](int64_t m) { return m <= smem_optin && m <= smem_sm - 2048; };
  bool packed = false;
  if (!fits(smem8)) {
    if (!fits(smem4) || stats[2] + 1 >= (1 << 13)) return cudaSuccess;  // does not fit: one-sweep form
    packed = true;
  }
  const int64_t smem = packed ? smem4 : smem8;
  P2CK(launch_scan(p.hhcount, p.hoff2, B, p.scan_tmp, st));
  P2CK(launch_scan(p.s2count, p.soff2, B, p.scan_tmp, st));
  P2CK(launch_scan(p.nslc, p.sloff2, B, p.scan_tmp, st));
  int32_t tot[3] = {0, 0, 0};
  P2CK(cudaMemcpyAsync(&tot[0], p.hoff2 + B, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  P2CK(cudaMemcpyAsync(&tot[1], p.soff2 + B, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  P2CK(cudaMemcpyAsync(&tot[2], p.sloff2 + B, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  P2CK(cudaStreamSynchronize(st));
  P2CK(grow2(&p.halo2, &p.halo2_cap, tot[0] > 0 ? tot[0] : 1));
  P2CK(grow2(&p.lec2, &p.lec2_cap, tot[1] > 0 ? tot[1] : 1));
  P2CK(grow2(&p.slc2, &p.slc2_cap, tot[2] > 0 ? tot[2] : 1));
  P2CK(grow2(&p.order2, &p.order2_cap, 32LL * (tot[2] > 0 ? tot[2] : 1)));
  const size_t map_smem = 2 * kSortCap2 * sizeof(int32_t);
  P2CK(cudaFuncSetAttribute(plan_map2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)map_smem));
  plan_map2_kernel<<<B, 512, map_smem, st>>>(p.irp, p.iec, p.part, p.tmp, p.hcount, p.tmp2, p.h2count,
                                             p.hoff2, p.soff2, p.sloff2, F, p.halo2, p.order2, p.slc2, p.lec2);
  count_launch();
  P2CK(cudaGetLastError());
  p.packed2 = false;
  if (packed) {  // 4-byte entries, if every cost is below the padding cost
    P2CK(grow2(&p.lec2p, &p.lec2p_cap, tot[1] > 0 ? tot[1] : 1));
    P2CK(cudaMemsetAsync(p.stats2, 0, sizeof(int32_t), st));
    plan_pack2_kernel<<<(tot[1] + 255) / 256 > 0 ? (tot[1] + 255) / 256 : 1, 256, 0, st>>>(
        p.lec2, tot[1], F, p.lec2p, p.stats2);
    count_launch();
    P2CK(cudaGetLastError());
    int32_t bad = 0;
    P2CK(cudaMemcpyAsync(&bad, p.stats2, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    P2CK(cudaStreamSynchronize(st));
    if (bad) return cudaSuccess;  // some cost too large to pack: one-sweep form
    p.packed2 = true;
  }
  p.maxS2 = stats[0];
  p.maxSl2 = stats[1];
  p.maxL2 = stats[2];
  p.maxHH2 = stats[3];
  p.smem2 = (size_t)smem;
  p.frac_bits2 = F;
  p.valid2 = true;
  return cudaSuccess;
}

cudaError_t launch_gdp_tiled2(GdpPlan& p, const int32_t* lam_in, int32_t shift, int64_t max_sweeps, GdpCtl* ctl,
                              long long* trace_b2, unsigned long long* trace_ch, int64_t trace_cap,
                              long long budget, const int32_t* bint, int32_t bmax, cudaStream_t st) {
  P2CK(gather_perm(lam_in, p.perm, p.n, p.ilam[0], st));
  const int mode = !bint ? 0 : (bmax < 8 ? 1 : 2);
  const bool tr = trace_cap > 0;
  const void* kerns[2][2][3] = {
      {{(const void*)gdp_tiled2_kernel<false, 0, false>, (const void*)gdp_tiled2_kernel<false, 1, false>,
        (const void*)gdp_tiled2_kernel<false, 2, false>},
       {(const void*)gdp_tiled2_kernel<true, 0, false>, (const void*)gdp_tiled2_kernel<true, 1, false>,
        (const void*)gdp_tiled2_kernel<true, 2, false>}},
      {{(const void*)gdp_tiled2_kernel<false, 0, true>, (const void*)gdp_tiled2_kernel<false, 1, true>,
        (const void*)gdp_tiled2_kernel<false, 2, true>},
       {(const void*)gdp_tiled2_kernel<true, 0, true>, (const void*)gdp_tiled2_kernel<true, 1, true>,
        (const void*)gdp_tiled2_kernel<true, 2, true>}}};
  const void* kern = kerns[p.packed2 ? 1 : 0][tr ? 1 : 0][mode];
  const void* lec = p.packed2 ? (const void*)p.lec2p : (const void*)p.lec2;
  int32_t F = p.frac_bits2;
  const int threads = mode == 0 ? 1024 : 512;
  P2CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem2));
  int per_sm = 0;
  P2CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, p.smem2));
  int dev = 0, sms = 0;
  P2CK(cudaGetDevice(&dev));
  P2CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if ((long long)per_sm * sms < p.B) return cudaErrorCooperativeLaunchTooLarge;
  long long ms = max_sweeps, tc = trace_cap;
  int32_t* l0 = p.ilam[0];
  int32_t* l1 = p.ilam[1];
  void* args[] = {(void*)&p.part, (void*)&p.hcount, (void*)&p.hoff2, (void*)&p.soff2, (void*)&p.sloff2,
                  (void*)&p.halo2, (void*)&p.order2, (void*)&p.slc2, (void*)&lec, (void*)&l0, (void*)&l1,
                  (void*)&shift, (void*)&ms, (void*)&ctl, (void*)&trace_b2, (void*)&trace_ch, (void*)&tc,
                  (void*)&budget, (void*)&p.maxS2, (void*)&p.maxSl2, (void*)&p.maxL2, (void*)&p.maxHH2,
                  (void*)&bint, (void*)&F};
  cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(p.B), dim3(threads), args, p.smem2, st);
  count_launch();
  return e;
}

}  // namespace f2m
