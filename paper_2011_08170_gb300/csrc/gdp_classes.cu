// Class-by-class (Gauss-Seidel) GDP phase and the colouring it runs on.
//
// Section 5.1 updates every node from the same lambda (Jacobi, gdp.cu).  This
// variant updates one colour class at a time, a class being an independent
// set of the candidate graph: nodes of a class share no edge, so they update
// in parallel without interacting, each from the CURRENT lambda of its
// neighbours.  With the full step (shift = 1) every class update maximises the
// Lagrangian over that class's duals with the others fixed (block coordinate
// ascent), so the bound never decreases.  The paper does not describe this
// variant; it is an extension of the parallel update.
//
// Colouring: the greedy colouring in priority order -- each node takes the
// smallest colour not held by a neighbour of higher priority -- where priority
// is larger degree, then larger h(v), then smaller id, and h(v) is the first
// output of SplitMix64 (Steele, Lea and Flood 2014) seeded with v.  It is
// computed by Jones-Plassmann rounds (Jones and Plassmann 1993): in a round,
// every uncoloured node whose uncoloured neighbours all have lower priority
// takes the smallest colour absent from its coloured neighbours.  A node is
// coloured only after all its higher-priority neighbours and before all its
// lower-priority ones, so the result equals the sequential greedy colouring.
//
// Sweep (one persistent cooperative kernel): for class 0, 1, ..., C-1, every
// node of the class updates lambda in place (Eq. 9, Eq. 10 or its b_v form),
// then a device-wide barrier.  C barriers per sweep (C + 1 while the per-sweep
// bound is traced: the bound at the sweep's input needs a pass of its own).
// A node whose new value would reach |lambda| >= 2^29 keeps its value and the
// phase stops after that sweep.
#include <climits>
#include <vector>

#include "f2m_device.cuh"
#include "f2m_internal.h"
#include "gdp_rows.cuh"

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

// SplitMix64: one output from state `seed` (add the Weyl increment, then mix)
__device__ __forceinline__ unsigned long long splitmix64_first(unsigned long long seed) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// true if node u (degree du, hash hu) comes before node v in the colouring order
__device__ __forceinline__ bool higher_priority(int u, int du, unsigned long long hu, int v, int dv,
                                                unsigned long long hv) {
  if (du != dv) return du > dv;
  if (hu != hv) return hu > hv;
  return u < v;
}

__global__ void jp_round_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                int32_t n, int32_t* color, unsigned int* left,
                                unsigned int* ncolors) {
  unsigned waiting = 0;
  F2M_GRID_STRIDE(v, n) {
    if (color[v] >= 0) continue;
    const int beg = rp[v], end = rp[v + 1];
    const int dv = end - beg;
    const unsigned long long hv = splitmix64_first((unsigned long long)v);
    bool ready = true;
    for (int e = beg; e < end && ready; ++e) {
      const int u = ec[e].x;
      if (__ldcg(color + u) < 0) {
        const int du = rp[u + 1] - rp[u];
        if (higher_priority(u, du, splitmix64_first((unsigned long long)u), (int)v, dv, hv)) ready = false;
      }
    }
    if (!ready) {
      ++waiting;
      continue;
    }
    // smallest colour absent from the coloured neighbours, 64 colours at a time
    int c = -1;
    for (int base = 0; c < 0; base += 64) {
      unsigned long long used = 0;
      for (int e = beg; e < end; ++e) {
        const int k = __ldcg(color + ec[e].x) - base;
        if (k >= 0 && k < 64) used |= 1ull << k;
      }
      if (~used) c = base + __ffsll((long long)~used) - 1;
    }
    color[v] = c;
    atomicMax(ncolors, (unsigned int)(c + 1));
  }
  waiting = warp_sum_u(waiting);
  if ((threadIdx.x & 31) == 0 && waiting) atomicAdd(left, waiting);
}

__global__ void class_count_kernel(const int32_t* __restrict__ color, int32_t n, int32_t* count) {
  F2M_GRID_STRIDE(v, n) atomicAdd(count + color[v], 1);
}

// order[off[c] + k] = the k-th node of class c placed (order within a class is
// arbitrary: its nodes do not interact)
__global__ void class_scatter_kernel(const int32_t* __restrict__ color, int32_t n,
                                     const int32_t* __restrict__ off, int32_t* cursor,
                                     int32_t* order) {
  F2M_GRID_STRIDE(v, n) {
    const int c = color[v];
    order[off[c] + atomicAdd(cursor + c, 1)] = (int32_t)v;
  }
}

cudaError_t color_classes(const int32_t* rp, const int2* ec, int32_t n, ClassPlan& cp,
                          cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (cp.cap < n) {
    if (cp.color) dev_free(cp.color);
    if (cp.order) dev_free(cp.order);
    if (cp.ctl) dev_free(cp.ctl);
    cp.color = cp.order = nullptr;
    cp.ctl = nullptr;
    cp.cap = 0;
    e = dev_malloc((void**)&cp.color, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = dev_malloc((void**)&cp.order, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = dev_malloc((void**)&cp.ctl, sizeof(unsigned int) * 2);
    if (e != cudaSuccess) return e;
    cp.cap = n;
  }
  e = cudaMemsetAsync(cp.color, 0xFF, sizeof(int32_t) * n, st);  // -1: uncoloured
  if (e == cudaSuccess) e = cudaMemsetAsync(cp.ctl, 0, sizeof(unsigned int) * 2, st);
  if (e != cudaSuccess) return e;
  // rounds until no node waits; each round colours at least the uncoloured
  // node of highest priority, so there are at most n rounds
  unsigned int h[2] = {1, 0};
  for (int32_t round = 0; h[0] > 0; ++round) {
    if (round >= n) return cudaErrorUnknown;
    e = cudaMemsetAsync(cp.ctl, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    jp_round_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp, ec, n, cp.color, cp.ctl, cp.ctl + 1);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cp.ctl, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    cp.rounds = round + 1;
  }
  const int32_t C = (int32_t)h[1];
  // class offsets: counts on the device, prefix sums on the host (C is small)
  if (cp.off) dev_free(cp.off);
  cp.off = nullptr;
  int32_t* d_tmp = nullptr;
  e = dev_malloc((void**)&cp.off, sizeof(int32_t) * (C + 1));
  if (e == cudaSuccess) e = dev_malloc((void**)&d_tmp, sizeof(int32_t) * (C + 1));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_tmp, 0, sizeof(int32_t) * (C + 1), st);
  if (e == cudaSuccess) {
    class_count_kernel<<<grid_for(n, 256), 256, 0, st>>>(cp.color, n, d_tmp);
    count_launch();
    e = cudaGetLastError();
  }
  std::vector<int32_t> cnt(C + 1, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_tmp, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    cp.h_off.assign(C + 1, 0);
    for (int32_t c = 0; c < C; ++c) cp.h_off[c + 1] = cp.h_off[c] + cnt[c];
    e = cudaMemcpyAsync(cp.off, cp.h_off.data(), sizeof(int32_t) * (C + 1), cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(d_tmp, 0, sizeof(int32_t) * (C + 1), st);
  if (e == cudaSuccess) {
    class_scatter_kernel<<<grid_for(n, 256), 256, 0, st>>>(cp.color, n, cp.off, d_tmp, cp.order);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d_tmp) dev_free(d_tmp);
  if (e != cudaSuccess) return e;
  cp.ncolors = C;
  return cudaSuccess;
}

void class_plan_free(ClassPlan& cp) {
  if (cp.color) dev_free(cp.color);
  if (cp.order) dev_free(cp.order);
  if (cp.off) dev_free(cp.off);
  if (cp.ctl) dev_free(cp.ctl);
  cp = ClassPlan{};
}

// MODE: see row_order_pair (gdp_rows.cuh)
template <int G, int MODE>
__global__ void __launch_bounds__(512)
gdp_classes_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                   const int32_t* __restrict__ bdeg, int32_t* lam,
                   const int32_t* __restrict__ order, const int32_t* __restrict__ off,
                   int32_t ncolors, int32_t n, int32_t F, int32_t shift, long long max_sweeps,
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
    long long b2 = 0;
    unsigned ch = 0;
    int ovf = 0;
    bool ok = true;
    if (t < trace_cap) {
      // the bound at the sweep's input: 2 * b_v * lambda_v + sum of min(0, z)
      for (long long v = gid; v < n; v += ngroups) {
        const int beg = __ldg(rp + v), end = __ldg(rp + v + 1);
        const int lv = ld_cg(lam + v);
        int z1, z2;
        const int bv = row_order_pair<G, MODE>(ec, lam, bdeg, v, beg, end, sub, gmask, lv, F, b2, z1, z2);
        if (sub == 0) b2 += 2LL * bv * lv;
      }
      ok = grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, budget);
    }
    for (int c = 0; c < ncolors && ok; ++c) {
      const int i0 = __ldg(off + c), i1 = __ldg(off + c + 1);
      for (long long i = i0 + gid; i < i1; i += ngroups) {
        const int v = __ldg(order + i);
        const int beg = __ldg(rp + v), end = __ldg(rp + v + 1);
        const int lv = ld_cg(lam + v);
        long long unused = 0;
        int z1, z2;
        row_order_pair<G, MODE>(ec, lam, bdeg, v, beg, end, sub, gmask, lv, F, unused, z1, z2);
        if (sub == 0) {
          const long long d = gdp_step(z1, z2, shift);  // Eq. 10 (Eq. 8), truncated toward 0
          const long long nl = (long long)lv + d;
          ch += (d != 0);
          if (nl >= kLamLimit || nl <= -kLamLimit) ovf = 1;  // keeps its value
          else lam[v] = (int32_t)nl;
        }
      }
      if (c + 1 < ncolors) ok = grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, budget);
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
        if (x) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->slot_b2[s]), (unsigned long long)x);
        if (y) atomicAdd(&ctl->slot_ch[s], (unsigned long long)y);
        if (o) atomicOr(&ctl->status, kGdpOverflow);
        if (!ok) atomicOr(&ctl->status, kGdpTimeout);
      }
    }
    if (ok) ok = grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, budget);
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
      s_stop = (st != 0) || (chg == 0) || !ok;
    }
    __syncthreads();
    if (s_stop) break;
  }
}

template <int G, int MODE>
static cudaError_t launch_classes_g(const int32_t* rp, const int2* ec, const int32_t* bdeg,
                                    int32_t* lam, const ClassPlan& cp, int32_t n, int32_t F,
                                    int32_t shift, int64_t max_sweeps, GdpCtl* ctl,
                                    long long* trace_b2, unsigned long long* trace_ch,
                                    int64_t trace_cap, long long budget, int num_sms,
                                    cudaStream_t st) {
  const int threads = 512;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, gdp_classes_kernel<G, MODE>, threads, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if (per_sm > 2) per_sm = 2;
  int grid = num_sms * per_sm;
  long long max_grid = ((long long)n * G + threads - 1) / threads;
  if (max_grid < 1) max_grid = 1;
  if (grid > max_grid) grid = (int)max_grid;
  long long ms = max_sweeps;
  long long tc = trace_cap;
  const int32_t* order = cp.order;
  const int32_t* off = cp.off;
  int32_t C = cp.ncolors;
  void* args[] = {(void*)&rp,    (void*)&ec,    (void*)&bdeg,     (void*)&lam,
                  (void*)&order, (void*)&off,   (void*)&C,        (void*)&n,
                  (void*)&F,     (void*)&shift, (void*)&ms,       (void*)&ctl,
                  (void*)&trace_b2, (void*)&trace_ch, (void*)&tc, (void*)&budget};
  err = cudaLaunchCooperativeKernel((const void*)gdp_classes_kernel<G, MODE>, dim3(grid),
                                    dim3(threads), args, 0, st);
  count_launch();
  return err;
}

cudaError_t launch_gdp_classes(const int32_t* rp, const int2* ec, const int32_t* bdeg, int32_t bmax,
                               int32_t* lam, const ClassPlan& cp, int32_t n, int32_t F,
                               int32_t shift, int64_t max_sweeps, GdpCtl* ctl, long long* trace_b2,
                               unsigned long long* trace_ch, int64_t trace_cap, long long budget,
                               int num_sms, cudaStream_t st) {
  if (bdeg && bmax < kTopK)
    return launch_classes_g<4, 1>(rp, ec, bdeg, lam, cp, n, F, shift, max_sweeps, ctl, trace_b2,
                                  trace_ch, trace_cap, budget, num_sms, st);
  if (bdeg)
    return launch_classes_g<4, 2>(rp, ec, bdeg, lam, cp, n, F, shift, max_sweeps, ctl, trace_b2,
                                  trace_ch, trace_cap, budget, num_sms, st);
  return launch_classes_g<4, 0>(rp, ec, nullptr, lam, cp, n, F, shift, max_sweeps, ctl, trace_b2,
                                trace_ch, trace_cap, budget, num_sms, st);
}

}  // namespace f2m
