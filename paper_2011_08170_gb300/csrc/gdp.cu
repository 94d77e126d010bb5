// GDP phase: one persistent cooperative kernel, one device-wide barrier per sweep.
//
// One sweep (Section 4, Eq. 9 and Eq. 10; Section 5.1: every node in parallel,
// Jacobi -- each sweep reads only the previous lambda):
//   for every node v:  z_e = c_e * 2^F - lambda_v - lambda_{col(e)}   (Eq. 9)
//                      z(2) <= z(3): 2nd and 3rd smallest z in the row  (Eq. 10)
//                      delta_v = trunc((z(2) + z(3)) / 2^shift)
//                      lambda'_v = lambda_v + delta_v
//   bound2 = 4 * sum_v lambda_v + sum over entries of min(0, z_e)
//   changed = #{v : delta_v != 0}
// The phase ends after the first sweep with changed == 0 (a fixed point), after
// max_sweeps, on |lambda| >= 2^29, or when a barrier wait exceeds its budget.
//
// Mapping: G consecutive lanes own one node; lane j of the group streams
// entries beg+j, beg+j+G, ... (8-byte {col, cost} loads), keeps a private
// top-3, and the group merges top-3s with xor shuffles.  Reductions are
// integer, so the result does not depend on the order of the atomics.
//
// Degree requirements b_v (fractional b-matching, Section 3 with Eq. 8: the
// b_v-th and (b_v+1)-th smallest adjusted values replace the 2nd and 3rd, and
// the bound term is 2 * b_v * lambda_v): the kernel's DEG form reads b_v per
// node.  When every b_v < kTopK, each lane keeps its kTopK smallest values
// sorted in registers and the group merges them (bitonic, Batcher 1968);
// otherwise every row finds its two order statistics by counting, each lane
// testing its own entries against the whole row.
#include <climits>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

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

// MODE 0: b_v = 2 (Eq. 10, top-3); 1: b_v read per node, all b_v < kTopK
// (registers); 2: b_v read per node, any value (counting)
template <int G, int MODE>
__global__ void __launch_bounds__(512)
gdp_persistent_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                      const int32_t* __restrict__ bdeg, int32_t* lam0,
                      int32_t* lam1, int32_t n, int32_t F, int32_t shift, long long max_sweeps,
                      GdpCtl* ctl, long long* trace_b2, unsigned long long* trace_ch,
                      long long trace_cap, long long budget) {
  __shared__ long long s_b2[32];
  __shared__ unsigned s_ch[32];
  __shared__ int s_ovf[32];
  __shared__ int s_stop;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int sub = lane & (G - 1);
  const unsigned gmask = (G >= 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const long long per_block = blockDim.x / G;
  const long long gid = (long long)blockIdx.x * per_block + tid / G;
  const long long ngroups = (long long)gridDim.x * per_block;
  const int nwarps = blockDim.x >> 5;

  for (long long t = 0; t < max_sweeps; ++t) {
    const int32_t* lin = (t & 1) ? lam1 : lam0;
    int32_t* lout = (t & 1) ? lam0 : lam1;
    long long b2 = 0;
    unsigned ch = 0;
    int ovf = 0;
    for (long long v = gid; v < n; v += ngroups) {
      const int beg = __ldg(rp + v), end = __ldg(rp + v + 1);
      const int lv = ld_cg(lin + v);
      int b, c, bv = 2;
      if constexpr (MODE == 1) {
        bv = __ldg(bdeg + v);
        row_order_pair_topk<G>(ec, lin, beg, end, sub, gmask, lv, F, bv, b2, b, c);
      } else if constexpr (MODE == 2) {
        bv = __ldg(bdeg + v);
        row_order_pair_count<G>(ec, lin, beg, end, sub, gmask, lv, F, bv, b2, b, c);
      } else {
        int a = INT_MAX;
        b = INT_MAX;
        c = INT_MAX;
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
      }
      if (sub == 0) {
        const long long d = gdp_step(b, c, shift);  // Eq. 10 (Eq. 8), truncated toward 0
        const long long nl = (long long)lv + d;
        ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
        lout[v] = (int32_t)nl;
        ch += (d != 0);
        b2 += 2LL * bv * lv;
      }
    }
    // block reduction, one atomic per block into this sweep's slot
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
        const int s = (int)(t % 3);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->slot_b2[s]), (unsigned long long)x);
        if (y) atomicAdd(&ctl->slot_ch[s], (unsigned long long)y);
        if (o) atomicOr(&ctl->status, kGdpOverflow);
      }
    }
    const bool ok = grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, budget);
    if (tid == 0) {
      if (!ok) atomicOr(&ctl->status, kGdpTimeout);
      volatile GdpCtl* vc = ctl;
      const int s = (int)(t % 3);
      const unsigned long long chg = vc->slot_ch[s];
      const int st = vc->status;
      if (blockIdx.x == 0) {
        if (t < trace_cap) {
          trace_b2[t] = vc->slot_b2[s];
          trace_ch[t] = chg;
        }
        const int r = (int)((t + 2) % 3);  // read by everyone after the previous barrier
        vc->slot_b2[r] = 0;
        vc->slot_ch[r] = 0;
        vc->sweeps = t + 1;
        vc->fixed_point = (chg == 0);
      }
      s_stop = (st != 0) || (chg == 0);
    }
    __syncthreads();
    if (s_stop) break;
  }
}

template <int G, int MODE>
static cudaError_t launch_gdp_g(const int32_t* rp, const int2* ec, const int32_t* bdeg,
                                int32_t* lam0, int32_t* lam1,
                                int32_t n, int32_t F, int32_t shift, int64_t max_sweeps,
                                GdpCtl* ctl, long long* trace_b2, unsigned long long* trace_ch,
                                int64_t trace_cap, long long budget, int num_sms,
                                cudaStream_t st) {
  const int threads = 512;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, gdp_persistent_kernel<G, MODE>, threads, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if (per_sm > 2) per_sm = 2;
  int grid = num_sms * per_sm;
  long long max_grid = ((long long)n * G + threads - 1) / threads;
  if (max_grid < 1) max_grid = 1;
  if (grid > max_grid) grid = (int)max_grid;
  long long ms = max_sweeps;
  long long tc = trace_cap;
  void* args[] = {(void*)&rp, (void*)&ec, (void*)&bdeg, (void*)&lam0, (void*)&lam1, (void*)&n, (void*)&F,
                  (void*)&shift, (void*)&ms, (void*)&ctl, (void*)&trace_b2, (void*)&trace_ch,
                  (void*)&tc, (void*)&budget};
  err = cudaLaunchCooperativeKernel((const void*)gdp_persistent_kernel<G, MODE>, dim3(grid),
                                    dim3(threads), args, 0, st);
  count_launch();
  return err;
}

cudaError_t launch_gdp(const int32_t* rp, const int2* ec, const int32_t* bdeg, int32_t bmax,
                       int32_t* lam0, int32_t* lam1, int32_t n, int32_t F, int32_t shift,
                       int64_t max_sweeps, GdpCtl* ctl, long long* trace_b2,
                       unsigned long long* trace_ch, int64_t trace_cap, long long budget,
                       int num_sms, cudaStream_t st) {
  if (bdeg && bmax < kTopK)
    return launch_gdp_g<4, 1>(rp, ec, bdeg, lam0, lam1, n, F, shift, max_sweeps, ctl, trace_b2,
                              trace_ch, trace_cap, budget, num_sms, st);
  if (bdeg)
    return launch_gdp_g<4, 2>(rp, ec, bdeg, lam0, lam1, n, F, shift, max_sweeps, ctl, trace_b2,
                              trace_ch, trace_cap, budget, num_sms, st);
  return launch_gdp_g<4, 0>(rp, ec, nullptr, lam0, lam1, n, F, shift, max_sweeps, ctl, trace_b2,
                            trace_ch, trace_cap, budget, num_sms, st);
}

// ---- bound2 at a given lambda, and rule (7) extraction ------------------------

__global__ void bound_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                             const int32_t* __restrict__ bdeg, const int32_t* __restrict__ lam,
                             int32_t n, int32_t fb, long long* out) {
  __shared__ long long s[32];
  long long acc = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const long long lv = lam[v];
    acc += 2LL * (bdeg ? bdeg[v] : 2) * lv;
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      const int2 q = ec[e];
      const long long z = ((long long)q.y << fb) - lv - lam[q.x];
      if (z < 0) acc += z;
    }
  }
  acc = warp_sum_ll(acc);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long x = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0;
    x = warp_sum_ll(x);
    if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)x);
  }
}

cudaError_t launch_bound(const int32_t* rp, const int2* ec, const int32_t* bdeg, const int32_t* lam,
                         int32_t n, int32_t fb, long long* out, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(out, 0, sizeof(long long), st);
  if (err != cudaSuccess) return err;
  const int threads = 256;
  int blocks = (int)((n + threads - 1) / threads);
  if (blocks > 4096) blocks = 4096;
  bound_kernel<<<blocks, threads, 0, st>>>(rp, ec, bdeg, lam, n, fb, out);
  count_launch();
  return cudaGetLastError();
}

// x2_e = 2 if z_e < 0, 1 if z_e == 0, 0 if z_e > 0 (rule (7)); count rows not
// summing to 2 * b_v (4 for the fractional 2-matching)
__global__ void extract_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                               const int32_t* __restrict__ bdeg, const int32_t* __restrict__ lam,
                               int32_t n, int32_t fb, uint8_t* __restrict__ x2,
                               unsigned long long* bad) {
  unsigned nb = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const long long lv = lam[v];
    int s = 0;
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      const int2 q = ec[e];
      const long long z = ((long long)q.y << fb) - lv - lam[q.x];
      const int x = z < 0 ? 2 : (z == 0 ? 1 : 0);
      x2[e] = (uint8_t)x;
      s += x;
    }
    nb += (s != 2 * (bdeg ? bdeg[v] : 2));
  }
  nb = warp_sum_u(nb);
  if ((threadIdx.x & 31) == 0 && nb) atomicAdd(bad, (unsigned long long)nb);
}

cudaError_t launch_extract(const int32_t* rp, const int2* ec, const int32_t* bdeg, const int32_t* lam,
                           int32_t n, int32_t fb, uint8_t* x2, unsigned long long* bad,
                           cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
  if (err != cudaSuccess) return err;
  const int threads = 256;
  int blocks = (int)((n + threads - 1) / threads);
  if (blocks > 4096) blocks = 4096;
  extract_kernel<<<blocks, threads, 0, st>>>(rp, ec, bdeg, lam, n, fb, x2, bad);
  count_launch();
  return cudaGetLastError();
}

__global__ void halve_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int32_t n) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    out[v] = in[v] >> 1;  // arithmetic shift: floor
}

cudaError_t launch_halve(const int32_t* lam_in, int32_t* lam_out, int32_t n, cudaStream_t st) {
  const int threads = 256;
  int blocks = (int)((n + threads - 1) / threads);
  if (blocks > 4096) blocks = 4096;
  halve_kernel<<<blocks, threads, 0, st>>>(lam_in, lam_out, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
