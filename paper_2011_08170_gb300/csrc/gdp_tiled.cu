// GDP phase, shared-memory tiled form (the default path of f2m_gdp / f2m_solve).
//
// The sweep is the same Jacobi step as gdp.cu (Eq. 9, Eq. 10, Section 5.1):
//   z_e = c_e * 2^F - lambda_v - lambda_u,  delta_v = trunc((z(2) + z(3)) / 2^shift),
//   bound2 = 4 sum lambda + sum_e min(0, z_e),  changed = #{delta != 0},
// so every result is bit-identical to the streaming kernel and to the oracle.
// What differs is where the data lives:
//
//  * Nodes are renumbered once along a Morton (Z-order) curve of their
//    coordinates, so each CTA's contiguous node range is a compact patch of the
//    plane and most neighbours of its nodes are its own nodes.  Jacobi sweeps do
//    not depend on node order, so the renumbering changes no value.
//  * A "plan" gives each CTA a node range of balanced entry count, the sorted
//    list of distinct outside nodes its rows reference (its halo), and its
//    entries rewritten as {local index, cost}: local < own is an own node,
//    local >= own is halo slot local - own.
//  * The persistent kernel loads its entries, row offsets and own lambda into
//    shared memory once per phase.  Per sweep it reads from global memory only
//    the halo lambdas (one round of independent loads, ~1 L2 round trip), does
//    all other work in shared memory, and writes its own new lambdas with
//    coalesced stores.  The stop test for sweep t-1 is read at the start of
//    sweep t and applied after it, hiding that read behind the sweep; a sweep
//    computed after the stop condition is discarded (nothing is published).
#include <climits>
#include <vector>

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

// ---- spatial renumbering ---------------------------------------------------------

// key = segment * 2^40 + Morton code (bit b of x at position 2b, bit b of y at
// 2b+1; x, y < 2^20), so nodes stay grouped by segment (instance) and follow a
// Morton curve inside each
__global__ void morton_kernel(const int2* __restrict__ xy, int32_t n, const int32_t* __restrict__ seg_off,
                              int32_t nseg, uint64_t* key, int32_t* idx) {
  F2M_GRID_STRIDE(v, n) {
    const unsigned x = (unsigned)xy[v].x, y = (unsigned)xy[v].y;
    uint64_t code = 0;
#pragma unroll
    for (int b = 0; b < 20; ++b)
      code |= ((uint64_t)((x >> b) & 1u) << (2 * b)) | ((uint64_t)((y >> b) & 1u) << (2 * b + 1));
    int lo = 0, hi = nseg - 1;  // segment of v: last s with seg_off[s] <= v
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg_off[mid] <= v) lo = mid; else hi = mid - 1;
    }
    key[v] = ((uint64_t)lo << 40) | code;
    idx[v] = (int32_t)v;
  }
}

__global__ void invert_perm_kernel(const int32_t* __restrict__ perm, int32_t n, int32_t* inv) {
  F2M_GRID_STRIDE(i, n) inv[perm[i]] = (int32_t)i;
}

__global__ void internal_degree_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ perm,
                                       int32_t n, int32_t* ideg) {
  F2M_GRID_STRIDE(i, n) {
    const int v = perm[i];
    ideg[i] = rp[v + 1] - rp[v];
  }
}

__global__ void internal_rows_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                     const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                                     const int32_t* __restrict__ irp, int32_t n, int2* __restrict__ iec) {
  F2M_GRID_STRIDE(i, n) {
    const int v = perm[i];
    const int a = rp[v], cnt = rp[v + 1] - a, o = irp[i];
    for (int k = 0; k < cnt; ++k) {
      const int2 q = ec[a + k];
      iec[o + k] = make_int2(inv[q.x], q.y);
    }
  }
}

__global__ void gather_perm_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ perm,
                                   int32_t n, int32_t* __restrict__ dst) {
  F2M_GRID_STRIDE(i, n) dst[i] = src[perm[i]];
}

__global__ void scatter_perm_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ perm,
                                    int32_t n, int32_t* __restrict__ dst) {
  F2M_GRID_STRIDE(i, n) dst[perm[i]] = src[i];
}

// ---- plan --------------------------------------------------------------------------

// part[b] = smallest node whose row starts at or after b * nnz / B
__global__ void partition_kernel(const int32_t* __restrict__ irp, int32_t n, int32_t B, int32_t* part) {
  F2M_GRID_STRIDE(b, B + 1) {
    if (b == 0) { part[0] = 0; continue; }
    if (b == B) { part[B] = n; continue; }
    const long long target = (long long)irp[n] * b / B;
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (irp[mid] >= target) hi = mid; else lo = mid + 1;
    }
    part[b] = lo;
  }
}

// Degree-descending order of a CTA's own nodes (ties by local id), sorted in
// shared memory; key = (2047 - min(deg, 2047)) << 20 | local.
__device__ void sort_own_by_degree(const int32_t* __restrict__ irp, int lo, int own, int* s_key) {
  const int tid = threadIdx.x, T = blockDim.x;
  int P = 1;
  while (P < own) P <<= 1;
  for (int i = tid; i < P; i += T) {
    if (i < own) {
      const int d = irp[lo + i + 1] - irp[lo + i];
      s_key[i] = ((2047 - min(d, 2047)) << 20) | i;
    } else {
      s_key[i] = INT_MAX;
    }
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += T) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int a = s_key[i], c = s_key[ixj];
          const bool up = (i & k) == 0;
          if ((a > c) == up) { s_key[i] = c; s_key[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// Pass 1, one CTA per node range: the sorted distinct outside nodes (halo) go
// to tmp[E0, E0 + H); hcount[b] = H; scount[b] = sliced entry count.
// stats: [0] max own nodes, [1] max sliced entries, [2] max halo, [3] 1 if some
// CTA does not fit the sort buffer (the tiled form is then off).
__global__ void plan_halo_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                 const int32_t* __restrict__ part, int32_t sort_cap,
                                 int32_t* __restrict__ tmp, int32_t* __restrict__ hcount,
                                 int32_t* __restrict__ scount, int32_t* __restrict__ stats) {
  extern __shared__ int s_sort[];
  __shared__ int s_cnt;
  __shared__ int s_warp[33];
  const int b = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int E0 = irp[lo], E1 = irp[hi];
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int e = E0 + tid; e < E1; e += T) {
    const int c = iec[e].x;
    if (c < lo || c >= hi) {
      const int k = atomicAdd(&s_cnt, 1);
      if (k < sort_cap) s_sort[k] = c;
    }
  }
  __syncthreads();
  const int m = s_cnt;
  if (m > sort_cap || own > sort_cap) {
    if (tid == 0) { atomicOr(&stats[3], 1); hcount[b] = 0; scount[b] = 0; }
    return;
  }
  int P = 1;
  while (P < m) P <<= 1;
  for (int i = m + tid; i < P; i += T) s_sort[i] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += T) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int a = s_sort[i], c = s_sort[ixj];
          const bool up = (i & k) == 0;
          if ((a > c) == up) { s_sort[i] = c; s_sort[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  // distinct values, compacted in order into tmp[E0, E0 + H)
  const int chunk = (m + T - 1) / T;
  const int i0 = min(m, tid * chunk), i1 = min(m, i0 + chunk);
  int cnt = 0;
  for (int i = i0; i < i1; ++i) cnt += (i == 0 || s_sort[i] != s_sort[i - 1]);
  int total = 0;
  int o = block_exclusive_scan(cnt, s_warp, total);
  for (int i = i0; i < i1; ++i)
    if (i == 0 || s_sort[i] != s_sort[i - 1]) tmp[E0 + o++] = s_sort[i];
  __syncthreads();
  // sliced size: 32 slots per slice, each slice as deep as its first (largest) row
  sort_own_by_degree(irp, lo, own, s_sort);
  int sz = 0;
  for (int s = tid; s * 32 < own; s += T) {
    const int first = s_sort[s * 32] & 0xFFFFF;
    sz += 32 * (irp[lo + first + 1] - irp[lo + first]);
  }
  int ssum = 0;
  block_exclusive_scan(sz, s_warp, ssum);
  if (tid == 0) {
    hcount[b] = total;
    scount[b] = ssum;
    atomicMax(&stats[0], own);
    atomicMax(&stats[1], ssum);
    atomicMax(&stats[2], total);
  }
}

// Pass 2: node order, slice table and sliced entries of each CTA.
//   order[lo + p]  = local node handled by slot p (degree-descending)
//   slc[lo + s]    = {offset of slice s in the CTA's entries, slice depth}
//   lec[soff[b] + base + k*32 + lane] = {local index, cost * 2^F} of entry k of
//   the node in slot 32 s + lane; short rows are padded with {zero slot, 2^30}.
__global__ void plan_map_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                const int32_t* __restrict__ part, const int32_t* __restrict__ tmp,
                                const int32_t* __restrict__ hoff, const int32_t* __restrict__ soff,
                                int32_t F, int32_t* __restrict__ halo, int32_t* __restrict__ order,
                                int2* __restrict__ slc, int2* __restrict__ lec) {
  extern __shared__ int s_key[];
  __shared__ int s_warp[33];
  const int b = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int E0 = irp[lo];
  const int hb = hoff[b], H = hoff[b + 1] - hb;
  const int zero_slot = own + H;
  const int32_t* list = tmp + E0;
  for (int h = tid; h < H; h += T) halo[hb + h] = list[h];
  sort_own_by_degree(irp, lo, own, s_key);
  const int nsl = (own + 31) / 32;
  // slice offsets: exclusive scan of 32 * depth over slices (chunked per thread)
  const int chunk = (nsl + T - 1) / T;
  const int s0 = min(nsl, tid * chunk), s1 = min(nsl, s0 + chunk);
  int sz = 0;
  for (int s = s0; s < s1; ++s) {
    const int first = s_key[s * 32] & 0xFFFFF;
    sz += 32 * (irp[lo + first + 1] - irp[lo + first]);
  }
  int total = 0;
  int base = block_exclusive_scan(sz, s_warp, total);
  for (int s = s0; s < s1; ++s) {
    const int first = s_key[s * 32] & 0xFFFFF;
    const int depth = irp[lo + first + 1] - irp[lo + first];
    slc[lo + s] = make_int2(base, depth);
    base += 32 * depth;
  }
  __syncthreads();
  int2* out = lec + soff[b];
  for (int p = tid; p < nsl * 32; p += T) {
    const int s = p >> 5, lane = p & 31;
    const int2 sl = slc[lo + s];
    if (p < own) {
      const int vl = s_key[p] & 0xFFFFF;
      order[lo + p] = vl;
      const int a = irp[lo + vl], d = irp[lo + vl + 1] - a;
      for (int k = 0; k < sl.y; ++k) {
        int2 q;
        if (k < d) {
          const int2 r = iec[a + k];
          int local;
          if (r.x >= lo && r.x < hi) {
            local = r.x - lo;
          } else {
            int x = 0, z = H;  // lower bound of r.x in the halo list
            while (x < z) {
              const int mid = (x + z) >> 1;
              if (list[mid] < r.x) x = mid + 1; else z = mid;
            }
            local = own + x;
          }
          q = make_int2(local, r.y << F);  // cost in units 2^-F
        } else {
          q = make_int2(zero_slot, 1 << 30);
        }
        out[sl.x + k * 32 + lane] = q;
      }
    } else {
      for (int k = 0; k < sl.y; ++k) out[sl.x + k * 32 + lane] = make_int2(zero_slot, 1 << 30);
    }
  }
}

// ---- the tiled persistent kernel ------------------------------------------------------

// BOUND: also sum the dual bound of every sweep (only traces need it)
template <bool BOUND>
__global__ void __launch_bounds__(1024, 1)
gdp_tiled_kernel(const int32_t* __restrict__ part, const int32_t* __restrict__ hoff,
                 const int32_t* __restrict__ soff, const int32_t* __restrict__ halo,
                 const int32_t* __restrict__ order, const int2* __restrict__ slc,
                 const int2* __restrict__ lec, int32_t* lam0, int32_t* lam1, int32_t* lam2,
                 int32_t shift, long long max_sweeps, GdpCtl* ctl, long long* trace_b2,
                 unsigned long long* trace_ch, long long trace_cap, long long budget, int32_t maxS,
                 int32_t maxO, int32_t maxH) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int maxSl = (maxO + 31) / 32;
  int2* s_lec = reinterpret_cast<int2*>(smem);            // sliced {local index, cost * 2^F}
  int2* s_slc = s_lec + maxS;                              // {offset, depth} per slice
  int* s_order = reinterpret_cast<int*>(s_slc + maxSl);    // node of each slot
  int* s_bufA = s_order + maxO;                            // [own lambda | halo lambda | 0]
  int* s_bufB = s_bufA + maxO + maxH + 1;
  int* s_hid = s_bufB + maxO + maxH + 1;                   // halo node ids
  __shared__ long long s_b2[32];
  __shared__ unsigned s_ch[32];
  __shared__ int s_ovf[32];
  __shared__ int s_stop;

  const int tid = threadIdx.x, T = blockDim.x, b = blockIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;

  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int hb = hoff[b], H = hoff[b + 1] - hb;
  const int S0 = soff[b], S = soff[b + 1] - S0;
  const int nsl = (own + 31) / 32;
  for (int e = tid; e < S; e += T) s_lec[e] = lec[S0 + e];
  for (int s = tid; s < nsl; s += T) s_slc[s] = slc[lo + s];
  for (int p = tid; p < own; p += T) s_order[p] = order[lo + p];
  for (int h = tid; h < H; h += T) s_hid[h] = halo[hb + h];
  for (int i = tid; i < own; i += T) s_bufA[i] = lam0[lo + i];
  if (tid == 0) {
    s_bufA[own + H] = 0;  // the zero slot padded entries point at
    s_bufB[own + H] = 0;
  }
  __syncthreads();

  volatile GdpCtl* vc = ctl;
  // Sweep t reads lambda from buffer t % 3 and publishes into (t + 1) % 3.
  // Its totals go to slot t % 4 after the block has arrived at barrier t, so
  // they are complete once barrier t + 1 has passed: sweep t + 2 reads them and
  // applies the stop test after its own work (that sweep and the one before
  // are then discarded: the first publishes nothing, the second published
  // values equal to its input at a fixed point and never overwrote the input
  // of an overflowing sweep, which lives in a third buffer).
  long long t = 0;
  bool natural_end = true;
  for (; t < max_sweeps; ++t) {
    int* s_in = (t & 1) ? s_bufB : s_bufA;   // own part holds lambda of sweep t
    int* s_out = (t & 1) ? s_bufA : s_bufB;
    const int r3 = (int)(t % 3);
    const int32_t* lin = r3 == 0 ? lam0 : (r3 == 1 ? lam1 : lam2);
    int32_t* lout = r3 == 0 ? lam1 : (r3 == 1 ? lam2 : lam0);
    unsigned long long pch = 1;
    int povf = 0;
    long long pb2 = 0;
    if (tid == 0 && t >= 2) {
      const int s = (int)((t - 2) % 4);
      pch = vc->q_ch[s];
      povf = vc->q_ovf[s];
      pb2 = vc->q_b2[s];
    }
    for (int h = tid; h < H; h += T) s_in[own + h] = ld_cg(lin + s_hid[h]);
    __syncthreads();

    long long b2 = 0;
    unsigned ch = 0;
    int ovf = 0;
    for (int p = tid; p < own; p += T) {
      const int2 sl = s_slc[p >> 5];
      const int vl = s_order[p];
      const int lv = s_in[vl];
      const int2* ent = s_lec + sl.x + (p & 31);
      int a = INT_MAX, bb = INT_MAX, c = INT_MAX, a1 = INT_MAX, b1 = INT_MAX, c1 = INT_MAX;
      long long neg = 0;
      int k = 0;
      for (; k + 1 < sl.y; k += 2) {  // two top-3 chains over alternate entries, merged
        const int2 q = ent[k * 32], q1 = ent[(k + 1) * 32];
        const int z = q.y - lv - s_in[q.x];  // Eq. 9
        const int z1 = q1.y - lv - s_in[q1.x];
        if (BOUND) neg += min(z, 0) + min(z1, 0);
        top3_insert_minmax(z, a, bb, c);
        top3_insert_minmax(z1, a1, b1, c1);
      }
      if (k < sl.y) {
        const int2 q = ent[k * 32];
        const int z = q.y - lv - s_in[q.x];
        if (BOUND) neg += min(z, 0);
        top3_insert_minmax(z, a, bb, c);
      }
      top3_merge(a1, b1, c1, a, bb, c);
      const long long d = gdp_step(bb, c, shift);  // Eq. 10, truncated toward 0
      const long long nl = (long long)lv + d;
      ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
      s_out[vl] = (int32_t)nl;
      ch += (d != 0);
      if (BOUND) b2 += neg + 4LL * lv;
    }
    // stop test for sweep t-2
    if (tid == 0) {
      int stop = 0;
      if (t >= 2) {
        stop = povf || (pch == 0);
        if (b == 0) {
          if (t - 2 < trace_cap) {
            trace_b2[t - 2] = pb2;
            trace_ch[t - 2] = pch;
          }
          if (stop) {
            vc->sweeps = t - 1;
            vc->fixed_point = (pch == 0) && !povf;
            if (povf) atomicOr(&ctl->status, kGdpOverflow);
          }
        }
      }
      if (b == 0) {  // slot (t+1) % 4 was last read during sweep t-1; next written in sweep t+1
        const int r = (int)((t + 1) % 4);
        vc->q_b2[r] = 0;
        vc->q_ch[r] = 0;
        vc->q_ovf[r] = 0;
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) { natural_end = false; break; }  // sweep t is discarded: nothing published
    for (int i = tid; i < own; i += T) lout[lo + i] = s_out[i];
    __syncthreads();
    if (tid == 0) grid_arrive_counted(&ctl->bar_count);

    // totals of sweep t, while the other blocks arrive
    b2 = warp_sum_ll(b2);
    ch = warp_sum_u(ch);
    ovf = __any_sync(0xffffffffu, ovf);
    if (lane == 0) { s_b2[warp] = b2; s_ch[warp] = ch; s_ovf[warp] = ovf; }
    __syncthreads();
    if (warp == 0) {
      long long x = lane < nwarps ? s_b2[lane] : 0;
      unsigned y = lane < nwarps ? s_ch[lane] : 0;
      int o = lane < nwarps ? s_ovf[lane] : 0;
      x = warp_sum_ll(x);
      y = warp_sum_u(y);
      o = __any_sync(0xffffffffu, o);
      if (lane == 0) {
        const int s = (int)(t % 4);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->q_b2[s]), (unsigned long long)x);
        if (y) atomicAdd(&ctl->q_ch[s], (unsigned long long)y);
        if (o) atomicOr(&ctl->q_ovf[s], 1);
        if (!grid_wait_counted(&ctl->bar_count, (unsigned)(t + 1) * gridDim.x, budget)) {
          atomicOr(&ctl->status, kGdpTimeout);
          s_stop = 1;
        } else {
          s_stop = 0;
        }
      }
    }
    __syncthreads();
    if (s_stop) { natural_end = false; break; }
  }
  if (natural_end) {
    // ran to the cap: one more barrier so the last sweep's totals are complete
    __syncthreads();
    if (tid == 0) grid_arrive_counted(&ctl->bar_count);
    if (tid == 0 && b == 0) {
      const bool ok = grid_wait_counted(&ctl->bar_count, (unsigned)(t + 1) * gridDim.x, budget);
      if (!ok) {
        atomicOr(&ctl->status, kGdpTimeout);
      } else {
        long long done = t;  // sweeps counted so far
        for (long long u = (t >= 2 ? t - 2 : 0); u < t; ++u) {
          const int s = (int)(u % 4);
          const unsigned long long chu = vc->q_ch[s];
          const int ovu = vc->q_ovf[s];
          if (u < trace_cap) {
            trace_b2[u] = vc->q_b2[s];
            trace_ch[u] = chu;
          }
          if (ovu || chu == 0) {
            done = u + 1;
            vc->fixed_point = (chu == 0) && !ovu;
            if (ovu) atomicOr(&ctl->status, kGdpOverflow);
            break;
          }
          vc->fixed_point = 0;
        }
        vc->sweeps = done;
      }
    }
  }
}

// ---- host side -----------------------------------------------------------------------

constexpr int kPlanSortCap = 16384;

template <typename T>
static cudaError_t grow(T** p, int64_t* cap, int64_t need) {
  if (*p && *cap >= need) return cudaSuccess;
  if (*p) dev_free(*p);
  *p = nullptr;
  *cap = 0;
  const int64_t c = need + (need >> 3) + 64;
  cudaError_t e = dev_malloc((void**)p, sizeof(T) * (size_t)c);
  if (e == cudaSuccess) *cap = c;
  return e;
}

void plan_free(GdpPlan& p) {
  void* ptrs[] = {p.perm, p.inv, p.irp, p.iec, p.lec, p.part, p.hoff, p.hcount, p.halo, p.tmp,
                  p.stats, p.ilam[0], p.ilam[1], p.ilam[2], p.keys, p.keys2, p.idx, p.sort_tmp,
                  p.scan_tmp, p.scount, p.soff, p.order, p.slc};
  for (void* q : ptrs)
    if (q) dev_free(q);
  p = GdpPlan();
}

#define PCK(x)                             \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

cudaError_t plan_renumber(const int2* xy, int32_t n, const std::vector<int32_t>& seg_off, GdpPlan& p,
                          cudaStream_t st) {
  int64_t cap = 0;
  const int32_t nseg = (int32_t)seg_off.size() - 1;
  int32_t* d_seg = nullptr;
  PCK(dev_malloc((void**)&d_seg, sizeof(int32_t) * seg_off.size()));
  cudaError_t e0 = cudaMemcpyAsync(d_seg, seg_off.data(), sizeof(int32_t) * seg_off.size(),
                                   cudaMemcpyHostToDevice, st);
  if (e0 != cudaSuccess) { dev_free(d_seg); return e0; }
  int end_bit = 40;
  while ((1LL << (end_bit - 40)) < nseg) ++end_bit;
  PCK(grow(&p.perm, &cap, n)); cap = 0;
  PCK(grow(&p.inv, &cap, n)); cap = 0;
  PCK(grow(&p.keys, &cap, n)); cap = 0;
  PCK(grow(&p.keys2, &cap, n)); cap = 0;
  PCK(grow(&p.idx, &cap, n));
  morton_kernel<<<grid_for(n, 256), 256, 0, st>>>(xy, n, d_seg, nseg, p.keys, p.idx);
  count_launch();
  cudaError_t e1 = cudaGetLastError();
  if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
  dev_free(d_seg);
  PCK(e1);
  size_t bytes = 0;
  PCK(sort_pairs_u64(nullptr, bytes, p.keys, p.keys2, p.idx, p.perm, n, end_bit, st));
  PCK(dev_malloc(&p.sort_tmp, bytes > 0 ? bytes : 1));
  PCK(sort_pairs_u64(p.sort_tmp, bytes, p.keys, p.keys2, p.idx, p.perm, n, end_bit, st));
  count_launch();
  invert_perm_kernel<<<grid_for(n, 256), 256, 0, st>>>(p.perm, n, p.inv);
  count_launch();
  PCK(cudaGetLastError());
  p.n = n;
  return cudaSuccess;
}

cudaError_t gather_perm(const int32_t* src, const int32_t* perm, int32_t n, int32_t* dst,
                        cudaStream_t st) {
  gather_perm_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, perm, n, dst);
  count_launch();
  return cudaGetLastError();
}

cudaError_t scatter_perm(const int32_t* src, const int32_t* perm, int32_t n, int32_t* dst,
                         cudaStream_t st) {
  scatter_perm_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, perm, n, dst);
  count_launch();
  return cudaGetLastError();
}

cudaError_t plan_build(const int32_t* rp, const int2* ec, int32_t n, int64_t nnz, int num_sms,
                       bool tiles, int32_t F, int32_t ctas_per_sm, GdpPlan& p, cudaStream_t st) {
  p.valid = false;
  p.version += 1;
  PCK(grow(&p.irp, &p.irp_cap, (int64_t)n + 1));
  PCK(grow(&p.iec, &p.iec_cap, nnz));
  PCK(grow(&p.tmp, &p.tmp_cap, nnz));
  PCK(grow(&p.ilam[0], &p.ilam_cap[0], n));
  PCK(grow(&p.ilam[1], &p.ilam_cap[1], n));
  PCK(grow(&p.ilam[2], &p.ilam_cap[2], n));
  PCK(grow(&p.scan_tmp, &p.scan_cap, (int64_t)scan_scratch_ints(n) + 1));
  // internal CSR: rows in renumbered order, columns renumbered
  int32_t* ideg = p.ilam[1];  // free until the phase starts
  internal_degree_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp, p.perm, n, ideg);
  count_launch();
  PCK(cudaGetLastError());
  PCK(launch_scan(ideg, p.irp, n, p.scan_tmp, st));
  internal_rows_kernel<<<grid_for(n, 128), 128, 0, st>>>(rp, ec, p.perm, p.inv, p.irp, n, p.iec);
  count_launch();
  PCK(cudaGetLastError());
  p.n = n;
  p.nnz = nnz;
  if (!tiles) return cudaSuccess;
  return plan_build_tiles(num_sms, F, ctas_per_sm, p, st);
}

cudaError_t plan_build_tiles(int num_sms, int32_t F, int32_t ctas_per_sm, GdpPlan& p, cudaStream_t st) {
  const int32_t n = p.n;
  p.valid = false;
  // per-CTA arrays, sized once for the largest grid (2 CTAs per SM)
  if (p.cta_cap < 2LL * num_sms + 1) {
    int32_t** arrs[] = {&p.part, &p.hcount, &p.scount, &p.soff, &p.hoff};
    for (int32_t** a : arrs) {
      if (*a) dev_free(*a);
      *a = nullptr;
      int64_t cap = 0;
      PCK(grow(a, &cap, 2LL * num_sms + 1));
    }
    p.cta_cap = 2LL * num_sms + 1;
  }
  // CTAs: 2 per SM x 512 threads, or 1 per SM x 1024 threads when a CTA's
  // shared memory would not fit twice on an SM
  int dev = 0, smem_optin = 0, smem_sm = 0;
  PCK(cudaGetDevice(&dev));
  PCK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PCK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  // Candidate shapes, tried in order: 1 CTA x 1024 threads per SM, then 2 CTAs
  // x 512 threads per SM (ctas_per_sm forces one).  Small graphs use fewer
  // CTAs (at least 8 nodes each).
  for (int attempt = 1; attempt < 3; ++attempt) {
    const int per_sm = attempt == 1 ? 1 : 2;
    const int threads = attempt == 1 ? 1024 : 512;
    if (ctas_per_sm != 0 && ctas_per_sm != per_sm) continue;
    int B = num_sms * per_sm;
    if ((int64_t)B > (int64_t)n / 8) B = (int)((int64_t)n / 8 > 1 ? (int64_t)n / 8 : 1);
    if (!p.stats) {
      int64_t cap = 0;
      PCK(grow(&p.stats, &cap, 4));
    }
    PCK(cudaMemsetAsync(p.stats, 0, 4 * sizeof(int32_t), st));
    partition_kernel<<<grid_for(B + 1, 256), 256, 0, st>>>(p.irp, n, B, p.part);
    count_launch();
    PCK(cudaGetLastError());
    const size_t sort_smem = kPlanSortCap * sizeof(int32_t);
    PCK(cudaFuncSetAttribute(plan_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem));
    plan_halo_kernel<<<B, 512, sort_smem, st>>>(p.irp, p.iec, p.part, kPlanSortCap, p.tmp, p.hcount,
                                                p.scount, p.stats);
    count_launch();
    PCK(cudaGetLastError());
    int32_t stats[4];
    PCK(cudaMemcpyAsync(stats, p.stats, sizeof(stats), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    if (stats[3]) return cudaSuccess;  // too many outside references: streaming kernel
    const int64_t maxSl = (stats[0] + 31) / 32;
    const int64_t smem = 8LL * stats[1] + 8LL * maxSl + 4LL * stats[0] +
                         8LL * (stats[0] + stats[2] + 1) + 4LL * stats[2];
    if (smem > smem_optin || smem * per_sm > smem_sm - 2048 * per_sm) continue;
    PCK(launch_scan(p.hcount, p.hoff, B, p.scan_tmp, st));
    PCK(launch_scan(p.scount, p.soff, B, p.scan_tmp, st));
    int32_t tot[2] = {0, 0};
    PCK(cudaMemcpyAsync(&tot[0], p.hoff + B, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(&tot[1], p.soff + B, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    const int32_t htot = tot[0];
    PCK(grow(&p.halo, &p.halo_cap, htot > 0 ? htot : 1));
    PCK(grow(&p.lec, &p.lec_cap, tot[1] > 0 ? tot[1] : 1));
    PCK(grow(&p.order, &p.order_cap, n));
    PCK(grow(&p.slc, &p.slc_cap, n));
    PCK(cudaFuncSetAttribute(plan_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem));
    plan_map_kernel<<<B, 512, sort_smem, st>>>(p.irp, p.iec, p.part, p.tmp, p.hoff, p.soff, F, p.halo,
                                               p.order, p.slc, p.lec);
    count_launch();
    PCK(cudaGetLastError());
    p.B = B;
    p.threads = threads;
    p.maxO = stats[0];
    p.maxS = stats[1];
    p.maxH = stats[2];
    p.smem = (size_t)smem;
    p.halo_total = htot;
    p.valid = true;
    return cudaSuccess;
  }
  return cudaSuccess;  // does not fit: streaming kernel
}

cudaError_t launch_gdp_tiled(GdpPlan& p, const int32_t* lam_in, int32_t shift, int64_t max_sweeps,
                             GdpCtl* ctl, long long* trace_b2, unsigned long long* trace_ch,
                             int64_t trace_cap, long long budget, cudaStream_t st) {
  PCK(gather_perm(lam_in, p.perm, p.n, p.ilam[0], st));
  const void* kern = trace_cap > 0 ? (const void*)gdp_tiled_kernel<true> : (const void*)gdp_tiled_kernel<false>;
  PCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  int per_sm = 0;
  PCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, p.threads, p.smem));
  int dev = 0, sms = 0;
  PCK(cudaGetDevice(&dev));
  PCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if ((long long)per_sm * sms < p.B) return cudaErrorCooperativeLaunchTooLarge;
  long long ms = max_sweeps, tc = trace_cap;
  int32_t* l0 = p.ilam[0];
  int32_t* l1 = p.ilam[1];
  int32_t* l2 = p.ilam[2];
  void* args[] = {(void*)&p.part, (void*)&p.hoff, (void*)&p.soff, (void*)&p.halo, (void*)&p.order,
                  (void*)&p.slc, (void*)&p.lec, (void*)&l0, (void*)&l1, (void*)&l2, (void*)&shift,
                  (void*)&ms, (void*)&ctl, (void*)&trace_b2, (void*)&trace_ch, (void*)&tc,
                  (void*)&budget, (void*)&p.maxS, (void*)&p.maxO, (void*)&p.maxH};
  cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(p.B), dim3(p.threads), args, p.smem, st);
  count_launch();
  return e;
}

cudaError_t plan_scatter_lambda(const GdpPlan& p, int which, int32_t* lam_out, cudaStream_t st) {
  return scatter_perm(p.ilam[which], p.perm, p.n, lam_out, st);
}

}  // namespace f2m
