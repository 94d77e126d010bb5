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

// Tiles: contiguous node ranges of one segment with at most TE entries and TN
// nodes (per kernel shape); tile k goes to CTA k mod G every sweep.
// Tile k's nodes are [tiles[k].x, tiles[k].y), its entries [tiles[k].w,
// tiles_e1[k]); the list holds only the tiles of instances still active when
// the launch was prepared (a phase is run as several launches, each over a
// fresh list, so that the tiles of converged instances stop taking turns).
//
// A tile's {col, cost} entries and row offsets are moved into shared memory by
// the bulk-copy engine (cp.async.bulk, completion counted in bytes on an
// mbarrier), S stages deep: while the CTA works on one tile the next S-1 are in
// flight.  The copies do not depend on lambda, so the issuing thread runs ahead
// across the end of a sweep (the grid barrier) into the next one.  Per tile:
// (1) all threads form w_e = c_e 2^F - lambda_u (lambda gathered from L2) into
// shared memory, (2) one thread per node takes the top-3 of w_e - lambda_v
// (Eq. 9) and applies Eq. 10.  Segments that changed nothing in sweep t are
// frozen by block 0 after barrier t; a CTA may still run a frozen segment's
// tile once more from a stale flag, which rewrites the same fixed point.
// bytes of one copy stage: entries and row offsets, each rounded out to 16 bytes
__host__ __device__ constexpr int stage_ec_bytes(int te) { return (te + 2) * 8; }
__host__ __device__ constexpr int stage_rp_bytes(int tn) { return (tn + 8) * 4; }
__host__ __device__ constexpr int stage_bytes(int te, int tn) { return stage_ec_bytes(te) + stage_rp_bytes(tn); }

__device__ __forceinline__ void mbar_init1(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait: false after `limit` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try(mbar, parity)) return true;
  return false;
}
// L2 policies: the CSR stream (larger than L2, read once per sweep) is evicted
// first so that lambda, gathered at random within an instance, stays resident
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar,
                                         uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar), "l"(pol)
      : "memory");
}
// lambda load that bypasses L1 (other SMs rewrite it between sweeps) and is kept in L2
__device__ __forceinline__ int ld_lam(const int32_t* p, uint64_t pol) {
  int v;
  asm volatile("ld.global.cg.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}

constexpr long long kBulkWaitLimit = 1LL << 24;

template <int T, int S, int TE, int TN, int MINB>
__global__ void __launch_bounds__(T, MINB)
gdp_batch_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                 const int4* __restrict__ tiles, const int32_t* __restrict__ tiles_e1,
                 const BatchChunk* __restrict__ chunk, int32_t nseg, uint8_t* active,
                 unsigned long long* seg_ch, long long* seg_sweeps, int32_t* lam0, int32_t* lam1,
                 int32_t F, int32_t shift, GdpCtl* ctl, long long budget, int32_t mcap) {
  const int32_t ntiles = chunk->ntiles;
  const long long t_base = chunk->t_base, max_sweeps = chunk->max_sweeps;
  // Software pipeline over the CTA's tiles: while the top-3 phase of tile j
  // runs, the lambda gathers of tile j+1 (same sweep) are in flight, and the
  // copies of tiles j+2 .. j+S-1 are landing.
  static_assert(S >= 3, "the look-ahead tile needs a copy issued one tile earlier");
  constexpr int kStageEcBytes = stage_ec_bytes(TE);
  constexpr int kStageBytes = stage_bytes(TE, TN);
  constexpr int KE = (TE + T - 1) / T;  // entries per thread in phase 1
  constexpr int KN = (TN + T - 1) / T;  // own lambdas per thread in phase 1
  static_assert(kStageBytes % 16 == 0 && kStageEcBytes % 16 == 0, "stage alignment");
  static_assert((2 * TE + 2 * TN) % 4 == 0, "tile table alignment");
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ unsigned s_tot[32];
  __shared__ int s_ovf[32];
  __shared__ unsigned s_tile_ch[2];  // changed counts of tiles j and j+1 (by j & 1)
  __shared__ int s_stop, s_abort, s_hdr[S];
  __shared__ __align__(8) unsigned long long s_full[S];
  const int tid = threadIdx.x, b = blockIdx.x, G = gridDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = T / 32;
  volatile GdpCtl* vc = ctl;
  volatile uint8_t* vact = active;

  int* s_w = reinterpret_cast<int*>(smem + S * kStageBytes);  // [2][TE] w of a prepared tile
  int* s_lv = s_w + 2 * TE;                                     // [2][TN] its own lambdas
  int4* s_mt = reinterpret_cast<int4*>(s_lv + 2 * TN);
  int* s_me1 = reinterpret_cast<int*>(s_mt + mcap);
  uint8_t* s_act = reinterpret_cast<uint8_t*>(s_me1 + mcap);
  const int my = b < ntiles ? (ntiles - 1 - b) / G + 1 : 0;  // tiles of this CTA

  for (int i = tid; i < my; i += T) {
    const int k = b + i * G;
    const int4 tl = tiles[k];
    s_mt[i] = tl;
    s_me1[i] = tiles_e1[k];
    s_act[i] = vact[tl.z];
  }
  if (tid == 0) {
    for (int st = 0; st < S; ++st) mbar_init1((uint32_t)__cvta_generic_to_shared(&s_full[st]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_stop = 0;
    s_abort = 0;
    s_tile_ch[0] = 0;
    s_tile_ch[1] = 0;
  }
  __syncthreads();

  const uint64_t pol_stream = policy_evict_first(), pol_lam = policy_evict_last();
  // The issuing thread is the CTA's last thread (rows go to the first nv
  // threads, so it usually has none): it issues while the others run phase 2.
  const bool issuer = tid == T - 1;
  int p_i = 0;  // issuing thread: next tile of its walk over (sweep, my tile)
  auto produce = [&](long long qq) {
    const int st = (int)(qq % S);
    for (;;) {
      if (p_i >= my) {  // end of a sweep
        s_hdr[st] = -1;
        p_i = 0;
        return;
      }
      const int i = p_i++;
      if (!s_act[i]) continue;
      const int4 tl = s_mt[i];
      const int e1 = s_me1[i];
      const int a0 = tl.w & ~1, a1 = (e1 + 1) & ~1;
      const int r0 = tl.x & ~3, r1 = (tl.y + 4) & ~3;
      const uint32_t ecb = (uint32_t)(a1 - a0) * 8u, rpb = (uint32_t)(r1 - r0) * 4u;
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&s_full[st]);
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem + st * kStageBytes);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(mb, ecb + rpb);
      bulk_g2s(dst, iec + a0, ecb, mb, pol_stream);
      bulk_g2s(dst + kStageEcBytes, irp + r0, rpb, mb, pol_stream);
      s_hdr[st] = i;
      return;
    }
  };

  long long q = 0;  // slots issued (issuing thread)
  if (issuer)
    for (; q < S - 1; ++q) produce(q);
  uint32_t phase_bits = 0;  // consumed uses of each stage, mod 2
  long long waited = 0;     // slots [0, waited) whose copies are known complete (or were END)
  // wait for the copy of slot sl (a tile); the result is the same in every thread
  auto wait_slot = [&](long long sl) -> bool {
    const int st = (int)(sl % S);
    const bool ok1 = mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&s_full[st]), (phase_bits >> st) & 1u,
                                       kBulkWaitLimit);
    const bool ok = __syncthreads_and(ok1) != 0;
    if (ok) {
      phase_bits ^= 1u << st;
      waited = sl + 1;
    }
    return ok;
  };
  int g[KE], c[KE], gl[KN];
  // phase 1, first half: the gathers of tile i from stage st into registers
  auto gather = [&](int i, int st, const int32_t* lin) {
    const int4 tl = s_mt[i];
    const int E0 = tl.w, ne = s_me1[i] - tl.w, v0 = tl.x, nv = tl.y - tl.x;
    const int2* sec = reinterpret_cast<const int2*>(smem + st * kStageBytes) + (E0 - (E0 & ~1));
#pragma unroll
    for (int k = 0; k < KE; ++k) {
      const int e = tid + k * T;
      if (e < ne) {
        const int2 w = sec[e];
        c[k] = w.y;
        g[k] = ld_lam(lin + w.x, pol_lam);
      }
    }
#pragma unroll
    for (int k = 0; k < KN; ++k) {
      const int v = tid + k * T;
      if (v < nv) gl[k] = ld_lam(lin + v0 + v, pol_lam);
    }
  };
  // phase 1, second half: w_e = c_e 2^F - lambda_u and the own lambdas into buffer bf
  auto settle = [&](int i, int bf) {
    const int4 tl = s_mt[i];
    const int ne = s_me1[i] - tl.w, nv = tl.y - tl.x;
    int* w = s_w + bf * TE;
    int* lv = s_lv + bf * TN;
#pragma unroll
    for (int k = 0; k < KE; ++k) {
      const int e = tid + k * T;
      if (e < ne) w[e] = (c[k] << F) - g[k];
    }
#pragma unroll
    for (int k = 0; k < KN; ++k) {
      const int v = tid + k * T;
      if (v < nv) lv[v] = gl[k];
    }
  };

  long long t = 0;
  unsigned ch = 0;
  int ovf = 0;
  bool prepared = false;  // slot j went through phase 1 (into buffer j & 1)
  __syncthreads();

  for (long long j = 0;; ++j) {
    const int st = (int)(j % S);
    const int i = s_hdr[st];
    const int32_t* lin = (t & 1) ? lam1 : lam0;
    int32_t* lout = (t & 1) ? lam0 : lam1;
    if (i >= 0) {
      const int bj = (int)(j & 1);
      if (!prepared) {  // first tile after a sweep boundary
        if (!wait_slot(j)) {
          if (tid == 0) s_abort = 1;
          break;
        }
        gather(i, st, lin);
        settle(i, bj);
        __syncthreads();
      }
      // look ahead: the next slot's copy was issued at least one tile ago
      const int st1 = (int)((j + 1) % S);
      const int i1 = s_hdr[st1];
      bool pre = false;
      if (i1 >= 0) {
        if (!wait_slot(j + 1)) {
          if (tid == 0) s_abort = 1;
          break;
        }
        gather(i1, st1, lin);
        pre = true;
      }
      if (issuer) produce(q++);  // slot j + S - 1 into the stage tile j - 1 freed
      // phase 2 of tile j: top-3 per row (Eq. 9), update (Eq. 10)
      const int4 tl = s_mt[i];
      const int v0 = tl.x, nv = tl.y - tl.x, E0 = tl.w;
      const int* srp = reinterpret_cast<const int*>(smem + st * kStageBytes + kStageEcBytes) + (v0 - (v0 & ~3));
      const int* w = s_w + bj * TE;
      const int* lvb = s_lv + bj * TN;
      unsigned tch = 0;
      for (int k = tid; k < nv; k += T) {
        const int lv = lvb[k];
        // two independent top-3 chains over alternate entries, merged (Eq. 9)
        int a = INT_MAX, bb = INT_MAX, cc = INT_MAX, a1 = INT_MAX, b1 = INT_MAX, c1 = INT_MAX;
        const int e_end = srp[k + 1] - E0;
        int e = srp[k] - E0;
        for (; e + 1 < e_end; e += 2) {
          top3_insert_minmax(w[e] - lv, a, bb, cc);
          top3_insert_minmax(w[e + 1] - lv, a1, b1, c1);
        }
        if (e < e_end) top3_insert_minmax(w[e] - lv, a, bb, cc);
        top3_merge(a1, b1, c1, a, bb, cc);
        const long long d = gdp_step(bb, cc, shift);  // Eq. 10, truncated toward 0
        const long long nl = (long long)lv + d;
        ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
        lout[v0 + k] = (int32_t)nl;
        tch += (d != 0);
      }
      if (pre) settle(i1, bj ^ 1);
      tch = __reduce_add_sync(0xffffffffu, tch);
      if (lane == 0 && tch) atomicAdd(&s_tile_ch[bj], tch);
      ch += (lane == 0) ? tch : 0;
      __syncthreads();
      // the count of tile j is complete; its slot is reset before any thread can
      // reach tile j + 2, which reuses it (tile j + 1 passes a barrier first)
      if (tid == 0) {
        if (s_tile_ch[bj]) atomicAdd(&seg_ch[(size_t)tl.z * 3 + (t % 3)], (unsigned long long)s_tile_ch[bj]);
        s_tile_ch[bj] = 0;
      }
      prepared = pre;
      continue;
    }
    // end of sweep t: totals, grid barrier, freezes, stop test
    if (issuer) produce(q++);
    prepared = false;
    if (waited == j) waited = j + 1;  // an END slot has no copy
    ch = warp_sum_u(ch);
    ovf = __any_sync(0xffffffffu, ovf);
    if (lane == 0) {
      s_tot[warp] = ch;
      s_ovf[warp] = ovf;
    }
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
    ch = 0;
    ovf = 0;
    bool stop = false;
    if (!grid_barrier_counted(&ctl->bar_count, (unsigned)(t + 1) * G, budget)) {
      if (tid == 0) atomicOr(&ctl->status, kGdpTimeout);
      stop = true;
    }
    if (b == 0 && !stop) {  // coordinator: freezes and slot resets for every segment
      for (int sgi = tid; sgi < nseg; sgi += T) {
        volatile unsigned long long* slot = seg_ch + (size_t)sgi * 3;
        if (vact[sgi] && slot[t % 3] == 0) {
          vact[sgi] = 0;
          seg_sweeps[sgi] = t_base + t + 1;
        }
        slot[(t + 2) % 3] = 0;
      }
    }
    for (int k = tid; k < my; k += T) s_act[k] = vact[s_mt[k].z];
    if (tid == 0) {
      const unsigned long long chg = vc->slot_ch[t % 3];
      const int stv = vc->status;
      if (b == 0) {
        vc->slot_ch[(t + 2) % 3] = 0;
        vc->sweeps = t + 1;
        vc->fixed_point = (chg == 0);
      }
      s_stop = stop || (stv != 0) || (chg == 0) || (t + 1 >= max_sweeps);
    }
    __syncthreads();
    if (s_stop) break;
    ++t;
  }
  if (s_abort && tid == 0) atomicOr(&ctl->status, kGdpTimeout);
  __syncthreads();
  // Wait (bounded) for the copies still in flight before the shared memory goes
  // away: every issued slot from `waited` on.  Consecutive slots use distinct
  // stages, and a stage's parity bit counts the uses already waited for.
  if (issuer) {
    for (long long sl = waited; sl < q; ++sl) {
      const int stg = (int)(sl % S);
      if (s_hdr[stg] < 0) continue;
      mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&s_full[stg]), (phase_bits >> stg) & 1u, kBulkWaitLimit);
      phase_bits ^= 1u << stg;
    }
  }
}

// Warp-tile form: every warp streams its own small tiles (tile k goes to warp
// k mod GW of the grid) through its own S copy stages, forms w_e in place in
// the stage (phase 1, lanes over entries) and takes the top-3 per row (phase
// 2, lanes over rows), synchronising only within the warp.  The warps of a CTA
// meet once per sweep, for the totals and the grid barrier.
template <int W, int S, int TE, int TN, int MINB>
__global__ void __launch_bounds__(W * 32, MINB)
gdp_batch_warp_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                      const int4* __restrict__ tiles, const int32_t* __restrict__ tiles_e1,
                      const BatchChunk* __restrict__ chunk, int32_t nseg, uint8_t* active,
                      unsigned long long* seg_ch, long long* seg_sweeps, int32_t* lam0, int32_t* lam1,
                      int32_t F, int32_t shift, GdpCtl* ctl, long long budget, int32_t mcap) {
  const int32_t ntiles = chunk->ntiles;
  const long long t_base = chunk->t_base, max_sweeps = chunk->max_sweeps;
  constexpr int kStageEcBytes = stage_ec_bytes(TE);
  constexpr int kStageBytes = stage_bytes(TE, TN);
  static_assert(kStageBytes % 16 == 0 && kStageEcBytes % 16 == 0, "stage alignment");
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ unsigned s_tot[W];
  __shared__ int s_ovf[W];
  __shared__ int s_stop, s_abort;
  __shared__ int s_hdr[W * S];
  __shared__ __align__(8) unsigned long long s_full[W * S];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int GW = gridDim.x * W, gw = blockIdx.x * W + warp;
  volatile GdpCtl* vc = ctl;
  volatile uint8_t* vact = active;

  uint8_t* my_stage = smem + (size_t)warp * S * kStageBytes;
  int4* s_mt = reinterpret_cast<int4*>(smem + (size_t)W * S * kStageBytes);  // [W][mcap]
  int* s_me1 = reinterpret_cast<int*>(s_mt + W * mcap);
  uint8_t* s_act = reinterpret_cast<uint8_t*>(s_me1 + W * mcap);
  const int my = gw < ntiles ? (ntiles - 1 - gw) / GW + 1 : 0;
  int4* m_mt = s_mt + warp * mcap;
  int* m_me1 = s_me1 + warp * mcap;
  uint8_t* m_act = s_act + warp * mcap;

  for (int i = lane; i < my; i += 32) {
    const int k = gw + i * GW;
    const int4 tl = tiles[k];
    m_mt[i] = tl;
    m_me1[i] = tiles_e1[k];
    m_act[i] = vact[tl.z];
  }
  if (lane == 0)
    for (int st = 0; st < S; ++st) mbar_init1((uint32_t)__cvta_generic_to_shared(&s_full[warp * S + st]));
  if (tid == 0) {
    s_stop = 0;
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const uint64_t pol_stream = policy_evict_first(), pol_lam = policy_evict_last();
  int p_i = 0;  // lane 0: next tile of this warp's walk over (sweep, my tile)
  auto produce = [&](long long q) {
    const int st = (int)(q % S);
    for (;;) {
      if (p_i >= my) {
        s_hdr[warp * S + st] = -1;  // end of a sweep
        p_i = 0;
        return;
      }
      const int i = p_i++;
      if (!m_act[i]) continue;
      const int4 tl = m_mt[i];
      const int e1 = m_me1[i];
      const int a0 = tl.w & ~1, a1 = (e1 + 1) & ~1;
      const int r0 = tl.x & ~3, r1 = (tl.y + 4) & ~3;
      const uint32_t ecb = (uint32_t)(a1 - a0) * 8u, rpb = (uint32_t)(r1 - r0) * 4u;
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&s_full[warp * S + st]);
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(my_stage + st * kStageBytes);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(mb, ecb + rpb);
      bulk_g2s(dst, iec + a0, ecb, mb, pol_stream);
      bulk_g2s(dst + kStageEcBytes, irp + r0, rpb, mb, pol_stream);
      s_hdr[warp * S + st] = i;
      return;
    }
  };

  long long q = 0;  // slots issued (lane 0)
  if (lane == 0)
    for (; q < S - 1; ++q) produce(q);
  __syncwarp();
  uint32_t phase_bits = 0;
  long long j = 0;          // first slot not consumed
  bool timed_out = false;   // the wait for slot j gave up
  unsigned ch_w = 0;        // lane 0: nodes changed by this warp in the sweep
  int ovf = 0;

  for (long long t = 0;; ++t) {
    const int32_t* lin = (t & 1) ? lam1 : lam0;
    int32_t* lout = (t & 1) ? lam0 : lam1;
    for (;;) {  // this warp's tiles of sweep t
      if (lane == 0) produce(q++);
      __syncwarp();
      const int st = (int)(j % S);
      const int i = s_hdr[warp * S + st];
      if (i < 0) {
        ++j;
        break;
      }
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&s_full[warp * S + st]);
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(mb, (phase_bits >> st) & 1u, kBulkWaitLimit));
      if (!ok) {
        timed_out = true;
        if (lane == 0) atomicOr(&s_abort, 1);
        break;
      }
      phase_bits ^= 1u << st;
      const int4 tl = m_mt[i];
      const int v0 = tl.x, nv = tl.y - tl.x, E0 = tl.w, ne = m_me1[i] - tl.w;
      int2* sec = reinterpret_cast<int2*>(my_stage + st * kStageBytes) + (E0 - (E0 & ~1));
      const int* srp = reinterpret_cast<const int*>(my_stage + st * kStageBytes + kStageEcBytes) + (v0 - (v0 & ~3));
#pragma unroll 4
      for (int e = lane; e < ne; e += 32) {  // w_e = c_e 2^F - lambda_u, in place of the column
        const int2 w = sec[e];
        sec[e].x = (w.y << F) - ld_lam(lin + w.x, pol_lam);
      }
      __syncwarp();
      unsigned chg = 0;
      for (int k = lane; k < nv; k += 32) {
        const int lv = ld_lam(lin + v0 + k, pol_lam);
        int a = INT_MAX, bb = INT_MAX, c = INT_MAX, a1 = INT_MAX, b1 = INT_MAX, c1 = INT_MAX;
        const int e_end = srp[k + 1] - E0;
        int e = srp[k] - E0;
        for (; e + 1 < e_end; e += 2) {  // Eq. 9, two chains over alternate entries
          top3_insert_minmax(sec[e].x - lv, a, bb, c);
          top3_insert_minmax(sec[e + 1].x - lv, a1, b1, c1);
        }
        if (e < e_end) top3_insert_minmax(sec[e].x - lv, a, bb, c);
        top3_merge(a1, b1, c1, a, bb, c);
        const long long d = gdp_step(bb, c, shift);  // Eq. 10, truncated toward 0
        const long long nl = (long long)lv + d;
        ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
        lout[v0 + k] = (int32_t)nl;
        chg += (d != 0);
      }
      chg = __reduce_add_sync(0xffffffffu, chg);
      __syncwarp();
      if (lane == 0 && chg) {
        atomicAdd(&seg_ch[(size_t)tl.z * 3 + (t % 3)], (unsigned long long)chg);
        ch_w += chg;
      }
      ++j;
    }
    // end of sweep t for the whole CTA: totals, grid barrier, freezes, stop test
    ovf = __any_sync(0xffffffffu, ovf);
    if (lane == 0) {
      s_tot[warp] = ch_w;
      s_ovf[warp] = ovf;
    }
    ch_w = 0;
    ovf = 0;
    __syncthreads();
    if (warp == 0) {
      unsigned y = lane < W ? s_tot[lane] : 0;
      int o = lane < W ? s_ovf[lane] : 0;
      y = __reduce_add_sync(0xffffffffu, y);
      o = __any_sync(0xffffffffu, o);
      if (lane == 0) {
        if (y) atomicAdd(&ctl->slot_ch[t % 3], (unsigned long long)y);
        if (o) atomicOr(&ctl->status, kGdpOverflow);
        if (s_abort) atomicOr(&ctl->status, kGdpTimeout);
      }
    }
    bool stop = s_abort != 0;
    if (!stop && !grid_barrier_counted(&ctl->bar_count, (unsigned)(t + 1) * gridDim.x, budget)) {
      if (tid == 0) atomicOr(&ctl->status, kGdpTimeout);
      stop = true;
    }
    if (blockIdx.x == 0 && !stop) {
      for (int sgi = tid; sgi < nseg; sgi += W * 32) {
        volatile unsigned long long* slot = seg_ch + (size_t)sgi * 3;
        if (vact[sgi] && slot[t % 3] == 0) {
          vact[sgi] = 0;
          seg_sweeps[sgi] = t_base + t + 1;
        }
        slot[(t + 2) % 3] = 0;
      }
    }
    for (int idx = tid; idx < W * mcap; idx += W * 32) {
      const int ww = idx / mcap, ii = idx % mcap;
      const int gww = blockIdx.x * W + ww;
      const int myw = gww < ntiles ? (ntiles - 1 - gww) / GW + 1 : 0;
      if (ii < myw) s_act[idx] = vact[s_mt[idx].z];
    }
    if (tid == 0) {
      const unsigned long long chg = vc->slot_ch[t % 3];
      const int stv = vc->status;
      if (blockIdx.x == 0) {
        vc->slot_ch[(t + 2) % 3] = 0;
        vc->sweeps = t + 1;
        vc->fixed_point = (chg == 0);
      }
      s_stop = stop || (stv != 0) || (chg == 0) || (t + 1 >= max_sweeps);
    }
    __syncthreads();
    if (s_stop) break;
  }
  // lane 0 waits (bounded) for this warp's copies still in flight: slots j..q-1
  if (lane == 0) {
    for (long long sl = j; sl < q; ++sl) {
      const int stg = (int)(sl % S);
      if (s_hdr[warp * S + stg] < 0) continue;
      mbar_wait_bounded((uint32_t)__cvta_generic_to_shared(&s_full[warp * S + stg]), (phase_bits >> stg) & 1u,
                        kBulkWaitLimit);
    }
  }
  (void)timed_out;
}

// Shapes of the batch kernel the autotuner picks from: threads per CTA, copy
// stages, CTAs per SM, tile entries, tile nodes, and whether tiles go to warps
// (gdp_batch_warp_kernel) or to CTAs (gdp_batch_kernel).
struct BatchShapeDef {
  int threads, stages, per_sm, te, tn, warp_tiles;
};
constexpr BatchShapeDef kBatchShapes[] = {
    {512, 3, 2, 2048, 768, 0},  {512, 3, 3, 1024, 384, 0},  {256, 3, 4, 1024, 384, 0},
    {256, 3, 6, 512, 192, 0},   {1024, 3, 1, 2048, 768, 0}, {256, 3, 3, 2048, 768, 0},
    {512, 4, 2, 1024, 384, 0},  {1024, 2, 1, 256, 96, 1},   {512, 2, 2, 256, 96, 1},
    {768, 3, 1, 256, 96, 1},    {512, 2, 1, 512, 176, 1},   {512, 3, 1, 256, 96, 1}};
constexpr int kNumBatchShapes = (int)(sizeof(kBatchShapes) / sizeof(kBatchShapes[0]));

template <int I>
static const void* batch_shape_ptr() {
  constexpr BatchShapeDef d = kBatchShapes[I];
  if constexpr (d.warp_tiles)
    return (const void*)gdp_batch_warp_kernel<d.threads / 32, d.stages, d.te, d.tn, d.per_sm>;
  else
    return (const void*)gdp_batch_kernel<d.threads, d.stages, d.te, d.tn, d.per_sm>;
}

static const void* batch_kernel_of(int shape) {
  switch (shape) {
    case 0: return batch_shape_ptr<0>();
    case 1: return batch_shape_ptr<1>();
    case 2: return batch_shape_ptr<2>();
    case 3: return batch_shape_ptr<3>();
    case 4: return batch_shape_ptr<4>();
    case 5: return batch_shape_ptr<5>();
    case 6: return batch_shape_ptr<6>();
    case 7: return batch_shape_ptr<7>();
    case 8: return batch_shape_ptr<8>();
    case 9: return batch_shape_ptr<9>();
    case 10: return batch_shape_ptr<10>();
    case 11: return batch_shape_ptr<11>();
  }
  return nullptr;
}
static_assert(kNumBatchShapes == 12, "one case per shape");

// dynamic shared memory: stages (per CTA, or per warp), the w buffer of the CTA
// form, and the tile table (int4 + int + flag per tile; per warp in the warp form)
static size_t batch_smem(int shape, int mcap) {
  const BatchShapeDef& d = kBatchShapes[shape];
  if (d.warp_tiles) {
    const int w = d.threads / 32;
    return (size_t)w * d.stages * stage_bytes(d.te, d.tn) + (size_t)w * mcap * 21 + 16;
  }
  return (size_t)d.stages * stage_bytes(d.te, d.tn) + (size_t)(2 * d.te + 2 * d.tn) * 4 + (size_t)mcap * 21 + 16;
}

// tile-table capacity per CTA (CTA form) or per warp (warp form)
static int32_t batch_mcap(int shape, int32_t ntiles, int32_t G) {
  const BatchShapeDef& d = kBatchShapes[shape];
  const long long units = d.warp_tiles ? (long long)G * (d.threads / 32) : G;
  long long m = (ntiles + units - 1) / units;
  return (int32_t)(m < 1 ? 1 : m);
}

int batch_shape_tile(int shape, int* te, int* tn) {
  if (shape < 0 || shape >= kNumBatchShapes) return 0;
  *te = kBatchShapes[shape].te;
  *tn = kBatchShapes[shape].tn;
  return 1;
}

int batch_num_shapes() { return kNumBatchShapes; }

int batch_shape_units(int shape) {
  if (shape < 0 || shape >= kNumBatchShapes) return 1;
  return kBatchShapes[shape].warp_tiles ? kBatchShapes[shape].threads / 32 : 1;
}

int batch_shape_blocks(int shape, int mcap) {
  if (shape < 0 || shape >= kNumBatchShapes) return 0;
  const void* k = batch_kernel_of(shape);
  const size_t sm = batch_smem(shape, mcap);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBatchShapes[shape].threads, sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm < kBatchShapes[shape].per_sm ? per_sm : kBatchShapes[shape].per_sm;
}

cudaError_t launch_gdp_batch(int shape, const int32_t* irp, const int2* iec, const int4* tiles,
                             const int32_t* tiles_e1, const BatchChunk* chunk, int32_t max_tiles, int32_t G,
                             int32_t nseg, uint8_t* active, unsigned long long* seg_ch, long long* seg_sweeps,
                             int32_t* lam0, int32_t* lam1, int32_t F, int32_t shift, GdpCtl* ctl,
                             long long budget, cudaStream_t st) {
  if (shape < 0 || shape >= kNumBatchShapes || G < 1) return cudaErrorInvalidValue;
  const int32_t mcap = batch_mcap(shape, max_tiles, G);
  const size_t sm = batch_smem(shape, mcap);
  const void* k = batch_kernel_of(shape);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&irp, (void*)&iec, (void*)&tiles, (void*)&tiles_e1, (void*)&chunk, (void*)&nseg,
                  (void*)&active, (void*)&seg_ch, (void*)&seg_sweeps, (void*)&lam0, (void*)&lam1,
                  (void*)&F, (void*)&shift, (void*)&ctl, (void*)&budget, (void*)&mcap};
  e = cudaLaunchCooperativeKernel(k, dim3(G), dim3(kBatchShapes[shape].threads), args, sm, st);
  count_launch();
  return e;
}

// dst[perm[i]] = (ctl->sweeps odd ? lam1 : lam0)[i]: the buffer a GDP launch
// ended in, chosen on the device so that no host decision is needed
__global__ void batch_scatter_final_kernel(const int32_t* __restrict__ lam0, const int32_t* __restrict__ lam1,
                                           const GdpCtl* ctl, const int32_t* __restrict__ perm, int32_t n,
                                           int32_t* __restrict__ dst) {
  const int32_t* src = (ctl->sweeps & 1) ? lam1 : lam0;
  F2M_GRID_STRIDE(i, n) dst[perm[i]] = src[i];
}

cudaError_t launch_batch_scatter_final(const int32_t* lam0, const int32_t* lam1, const GdpCtl* ctl,
                                       const int32_t* perm, int32_t n, int32_t* dst, cudaStream_t st) {
  batch_scatter_final_kernel<<<grid_for(n, 256), 256, 0, st>>>(lam0, lam1, ctl, perm, n, dst);
  count_launch();
  return cudaGetLastError();
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


// Copies the state of the instances flagged in done into the result arenas:
// one block per instance; lambda, its row offsets (kept absolute, as the
// caller reads them back relative to the first), and its {col, cost} and x
// entries to the arena offset eoff[s].
__global__ void batch_snapshot_kernel(const uint8_t* __restrict__ done, const int32_t* __restrict__ seg_off,
                                      const int32_t* __restrict__ rp, const int32_t* __restrict__ lam,
                                      const int2* __restrict__ ec, const uint8_t* __restrict__ x2,
                                      const long long* __restrict__ eoff, int32_t* res_lam, int32_t* res_rp,
                                      int2* res_ec, uint8_t* res_x2) {
  const int s = blockIdx.x;
  if (!done[s]) return;
  const int v0 = seg_off[s], ns = seg_off[s + 1] - v0;
  const int e0 = rp[v0], nz = rp[v0 + ns] - e0;
  const long long o = eoff[s];
  for (int i = threadIdx.x; i < ns; i += blockDim.x) res_lam[v0 + i] = lam[v0 + i];
  for (int i = threadIdx.x; i <= ns; i += blockDim.x) res_rp[v0 + s + i] = rp[v0 + i];
  for (int i = threadIdx.x; i < nz; i += blockDim.x) {
    res_ec[o + i] = ec[e0 + i];
    res_x2[o + i] = x2[e0 + i];
  }
}

cudaError_t launch_batch_snapshot(const uint8_t* done, const int32_t* seg_off, int32_t nseg, const int32_t* rp,
                                  const int32_t* lam, const int2* ec, const uint8_t* x2, const long long* eoff,
                                  int32_t* res_lam, int32_t* res_rp, int2* res_ec, uint8_t* res_x2,
                                  cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  batch_snapshot_kernel<<<nseg, 256, 0, st>>>(done, seg_off, rp, lam, ec, x2, eoff, res_lam, res_rp, res_ec,
                                              res_x2);
  count_launch();
  return cudaGetLastError();
}


// out[s] = rp[seg_off[s]] for s = 0..nseg: the first entry of every instance
__global__ void batch_seg_entry_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ seg_off,
                                       int32_t nseg, int32_t* out) {
  F2M_GRID_STRIDE(s, nseg + 1) out[s] = rp[seg_off[s]];
}

cudaError_t launch_batch_seg_entry(const int32_t* rp, const int32_t* seg_off, int32_t nseg, int32_t* out,
                                   cudaStream_t st) {
  batch_seg_entry_kernel<<<grid_for(nseg + 1, 256), 256, 0, st>>>(rp, seg_off, nseg, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
