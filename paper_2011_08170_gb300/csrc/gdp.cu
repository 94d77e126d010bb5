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
// the bound term is 2 * b_v * lambda_v): MODE 1 and 2 read b_v per node.  When
// every b_v < kTopK, each lane keeps its kTopK smallest values sorted in
// registers and the group merges them (bitonic, Batcher 1968); otherwise every
// row finds its two order statistics by counting, each lane testing its own
// entries against the whole row (gdp_rows.cuh).
#include <climits>

#include "f2m_device.cuh"
#include "f2m_internal.h"
#include "gdp_rows.cuh"

namespace f2m {

// MODE: see row_order_pair (gdp_rows.cuh)
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
      int b, c;
      const int bv = row_order_pair<G, MODE>(ec, lin, bdeg, v, beg, end, sub, gmask, lv, F, b2, b, c);
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

__global__ void double_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int32_t n) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    out[v] = 2 * in[v];  // |lambda| < 2^29: no overflow
}

cudaError_t launch_double(const int32_t* lam_in, int32_t* lam_out, int32_t n, cudaStream_t st) {
  const int threads = 256;
  int blocks = (int)((n + threads - 1) / threads);
  if (blocks > 4096) blocks = 4096;
  double_kernel<<<blocks, threads, 0, st>>>(lam_in, lam_out, n);
  count_launch();
  return cudaGetLastError();
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
