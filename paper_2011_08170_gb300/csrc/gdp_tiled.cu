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

// key = Morton code: bit b of x at position 2b, bit b of y at 2b+1 (x, y < 2^20)
__global__ void morton_kernel(const int2* __restrict__ xy, int32_t n, uint64_t* key, int32_t* idx) {
  F2M_GRID_STRIDE(v, n) {
    const unsigned x = (unsigned)xy[v].x, y = (unsigned)xy[v].y;
    uint64_t code = 0;
#pragma unroll
    for (int b = 0; b < 20; ++b)
      code |= ((uint64_t)((x >> b) & 1u) << (2 * b)) | ((uint64_t)((y >> b) & 1u) << (2 * b + 1));
    key[v] = code;
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

// stats: [0] max own nodes, [1] max entries, [2] max halo, [3] 1 if some CTA's
// outside references exceed the sort capacity (the tiled form is then off)
__global__ void plan_halo_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                 const int32_t* __restrict__ part, int32_t sort_cap,
                                 int32_t* __restrict__ tmp, int32_t* __restrict__ hcount,
                                 int32_t* __restrict__ stats) {
  extern __shared__ int s_sort[];
  __shared__ int s_cnt;
  __shared__ int s_warp[33];
  const int b = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lo = part[b], hi = part[b + 1];
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
  if (m > sort_cap) {
    if (tid == 0) { atomicOr(&stats[3], 1); hcount[b] = 0; }
    return;
  }
  int P = 1;
  while (P < m) P <<= 1;
  for (int i = m + tid; i < P; i += T) s_sort[i] = INT_MAX;
  __syncthreads();
  // bitonic sort of s_sort[0, P)
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
  if (tid == 0) {
    hcount[b] = total;
    atomicMax(&stats[0], hi - lo);
    atomicMax(&stats[1], E1 - E0);
    atomicMax(&stats[2], total);
  }
}

__global__ void plan_map_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                const int32_t* __restrict__ part, const int32_t* __restrict__ tmp,
                                const int32_t* __restrict__ hoff, int32_t* __restrict__ halo,
                                int2* __restrict__ lec) {
  const int b = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int E0 = irp[lo], E1 = irp[hi];
  const int hb = hoff[b], H = hoff[b + 1] - hb;
  const int32_t* list = tmp + E0;
  for (int h = tid; h < H; h += T) halo[hb + h] = list[h];
  for (int e = E0 + tid; e < E1; e += T) {
    const int2 q = iec[e];
    int local;
    if (q.x >= lo && q.x < hi) {
      local = q.x - lo;
    } else {
      int a = 0, z = H;  // lower bound of q.x in list[0, H)
      while (a < z) {
        const int mid = (a + z) >> 1;
        if (list[mid] < q.x) a = mid + 1; else z = mid;
      }
      local = own + a;
    }
    lec[e] = make_int2(local, q.y);
  }
}

// ---- the tiled persistent kernel ------------------------------------------------------

template <int G>
__global__ void __launch_bounds__(1024)
gdp_tiled_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ lec,
                 const int32_t* __restrict__ part, const int32_t* __restrict__ hoff,
                 const int32_t* __restrict__ halo, int32_t* lam0, int32_t* lam1, int32_t F,
                 int32_t shift, long long max_sweeps, GdpCtl* ctl, long long* trace_b2,
                 unsigned long long* trace_ch, long long trace_cap, long long budget, int32_t maxE,
                 int32_t maxO, int32_t maxH) {
  extern __shared__ __align__(16) unsigned char smem[];
  int2* s_lec = reinterpret_cast<int2*>(smem);
  int* s_rp = reinterpret_cast<int*>(s_lec + maxE);
  int* s_lamA = s_rp + maxO + 1;
  int* s_lamB = s_lamA + maxO;
  int* s_hl = s_lamB + maxO;
  int* s_hid = s_hl + maxH;
  __shared__ long long s_b2[32];
  __shared__ unsigned s_ch[32];
  __shared__ int s_ovf[32];
  __shared__ int s_stop;

  const int tid = threadIdx.x, T = blockDim.x, b = blockIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int sub = lane & (G - 1);
  const unsigned gmask = (G >= 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int ngroups = T / G, grp = tid / G;
  const long long div = 1LL << shift;

  const int lo = part[b], hi = part[b + 1], own = hi - lo;
  const int E0 = irp[lo], ents = irp[hi] - E0;
  const int hb = hoff[b], H = hoff[b + 1] - hb;
  for (int e = tid; e < ents; e += T) s_lec[e] = lec[E0 + e];
  for (int i = tid; i <= own; i += T) s_rp[i] = irp[lo + i] - E0;
  for (int h = tid; h < H; h += T) s_hid[h] = halo[hb + h];
  for (int i = tid; i < own; i += T) s_lamA[i] = lam0[lo + i];
  __syncthreads();

  volatile GdpCtl* vc = ctl;
  long long t = 0;
  for (; t < max_sweeps; ++t) {
    const int* s_in = (t & 1) ? s_lamB : s_lamA;
    int* s_out = (t & 1) ? s_lamA : s_lamB;
    const int32_t* lin = (t & 1) ? lam1 : lam0;
    int32_t* lout = (t & 1) ? lam0 : lam1;
    // the previous sweep's totals, complete since the last barrier; used after this sweep
    unsigned long long pch = 1;
    int pst = 0;
    long long pb2 = 0;
    if (tid == 0 && t > 0) {
      const int s = (int)((t - 1) % 3);
      pch = vc->slot_ch[s];
      pst = vc->status;
      pb2 = vc->slot_b2[s];
    }
    for (int h = tid; h < H; h += T) s_hl[h] = ld_cg(lin + s_hid[h]);
    __syncthreads();

    long long b2 = 0;
    unsigned ch = 0;
    int ovf = 0;
    for (int vl = grp; vl < own; vl += ngroups) {
      const int lv = s_in[vl];
      const int beg = s_rp[vl], end = s_rp[vl + 1];
      int a = INT_MAX, bb = INT_MAX, c = INT_MAX;
      for (int e = beg + sub; e < end; e += G) {
        const int2 q = s_lec[e];
        const int lu = q.x < own ? s_in[q.x] : s_hl[q.x - own];
        const int z = (q.y << F) - lv - lu;  // Eq. 9
        b2 += min(z, 0);
        top3_insert(z, a, bb, c);
      }
      if (G > 1) {
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
          const int pa = __shfl_xor_sync(gmask, a, o);
          const int pb = __shfl_xor_sync(gmask, bb, o);
          const int pc = __shfl_xor_sync(gmask, c, o);
          top3_insert(pa, a, bb, c);
          top3_insert(pb, a, bb, c);
          top3_insert(pc, a, bb, c);
        }
      }
      if (sub == 0) {
        const long long d = ((long long)bb + (long long)c) / div;  // Eq. 10, truncated toward 0
        const long long nl = (long long)lv + d;
        ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
        s_out[vl] = (int32_t)nl;
        ch += (d != 0);
        b2 += 4LL * lv;
      }
    }
    // decide about sweep t-1 now that this sweep's work has hidden the read
    if (tid == 0) {
      int stop = 0;
      if (t > 0) {
        stop = (pst != 0) || (pch == 0);
        if (b == 0) {
          if (t - 1 < trace_cap) {
            trace_b2[t - 1] = pb2;
            trace_ch[t - 1] = pch;
          }
          const int r = (int)((t + 1) % 3);  // last read during sweep t-1
          vc->slot_b2[r] = 0;
          vc->slot_ch[r] = 0;
          if (stop) {
            vc->sweeps = t;
            vc->fixed_point = (pch == 0) && (pst == 0);
          }
        }
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;  // sweep t is discarded: nothing published
    for (int i = tid; i < own; i += T) lout[lo + i] = s_out[i];

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
    if (!grid_barrier_counted(&ctl->bar_count, (unsigned)(t + 1) * gridDim.x, budget)) {
      if (tid == 0) atomicOr(&ctl->status, kGdpTimeout);
      break;
    }
  }
  if (t == max_sweeps && b == 0 && tid == 0) {  // ran to the cap: settle the last sweep
    if (t > 0) {
      const int s = (int)((t - 1) % 3);
      const unsigned long long pch = vc->slot_ch[s];
      if (t - 1 < trace_cap) {
        trace_b2[t - 1] = vc->slot_b2[s];
        trace_ch[t - 1] = pch;
      }
      vc->fixed_point = (pch == 0) && (vc->status == 0);
    }
    vc->sweeps = t;
  }
}

// ---- host side -----------------------------------------------------------------------

constexpr int kPlanSortCap = 16384;

template <typename T>
static cudaError_t grow(T** p, int64_t* cap, int64_t need) {
  if (*p && *cap >= need) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const int64_t c = need + (need >> 3) + 64;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)c);
  if (e == cudaSuccess) *cap = c;
  return e;
}

void plan_free(GdpPlan& p) {
  void* ptrs[] = {p.perm, p.inv, p.irp, p.iec, p.lec, p.part, p.hoff, p.hcount, p.halo, p.tmp,
                  p.stats, p.ilam[0], p.ilam[1], p.keys, p.keys2, p.idx, p.sort_tmp, p.scan_tmp};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p = GdpPlan();
}

#define PCK(x)                             \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

cudaError_t plan_renumber(const int2* xy, int32_t n, GdpPlan& p, cudaStream_t st) {
  int64_t cap = 0;
  PCK(grow(&p.perm, &cap, n)); cap = 0;
  PCK(grow(&p.inv, &cap, n)); cap = 0;
  PCK(grow(&p.keys, &cap, n)); cap = 0;
  PCK(grow(&p.keys2, &cap, n)); cap = 0;
  PCK(grow(&p.idx, &cap, n));
  morton_kernel<<<grid_for(n, 256), 256, 0, st>>>(xy, n, p.keys, p.idx);
  count_launch();
  PCK(cudaGetLastError());
  size_t bytes = 0;
  PCK(sort_pairs_u64(nullptr, bytes, p.keys, p.keys2, p.idx, p.perm, n, 40, st));
  PCK(cudaMalloc(&p.sort_tmp, bytes > 0 ? bytes : 1));
  PCK(sort_pairs_u64(p.sort_tmp, bytes, p.keys, p.keys2, p.idx, p.perm, n, 40, st));
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
                       bool tiles, GdpPlan& p, cudaStream_t st) {
  p.valid = false;
  p.version += 1;
  PCK(grow(&p.irp, &p.irp_cap, (int64_t)n + 1));
  PCK(grow(&p.iec, &p.iec_cap, nnz));
  PCK(grow(&p.lec, &p.lec_cap, nnz));
  PCK(grow(&p.tmp, &p.tmp_cap, nnz));
  PCK(grow(&p.ilam[0], &p.ilam_cap[0], n));
  PCK(grow(&p.ilam[1], &p.ilam_cap[1], n));
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
  if (!tiles) return cudaSuccess;

  // CTAs: 2 per SM x 512 threads, or 1 per SM x 1024 threads when a CTA's
  // shared memory would not fit twice on an SM
  int dev = 0, smem_optin = 0, smem_sm = 0;
  PCK(cudaGetDevice(&dev));
  PCK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PCK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  for (int attempt = 0; attempt < 2; ++attempt) {
    const int per_sm = attempt == 0 ? 2 : 1;
    const int threads = attempt == 0 ? 512 : 1024;
    int B = num_sms * per_sm;
    if ((int64_t)B > (int64_t)n / 8) B = (int)((int64_t)n / 8 > 1 ? (int64_t)n / 8 : 1);
    int64_t cap = 0;
    if (p.part) cudaFree(p.part);
    p.part = nullptr;
    PCK(grow(&p.part, &cap, B + 1)); cap = 0;
    if (p.hcount) cudaFree(p.hcount);
    p.hcount = nullptr;
    PCK(grow(&p.hcount, &cap, B + 1)); cap = 0;
    if (p.hoff) cudaFree(p.hoff);
    p.hoff = nullptr;
    PCK(grow(&p.hoff, &cap, B + 1));
    if (!p.stats) {
      cap = 0;
      PCK(grow(&p.stats, &cap, 4));
    }
    PCK(cudaMemsetAsync(p.stats, 0, 4 * sizeof(int32_t), st));
    partition_kernel<<<grid_for(B + 1, 256), 256, 0, st>>>(p.irp, n, B, p.part);
    count_launch();
    PCK(cudaGetLastError());
    const size_t sort_smem = kPlanSortCap * sizeof(int32_t);
    PCK(cudaFuncSetAttribute(plan_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem));
    plan_halo_kernel<<<B, 512, sort_smem, st>>>(p.irp, p.iec, p.part, kPlanSortCap, p.tmp, p.hcount, p.stats);
    count_launch();
    PCK(cudaGetLastError());
    int32_t stats[4];
    PCK(cudaMemcpyAsync(stats, p.stats, sizeof(stats), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    if (stats[3]) return cudaSuccess;  // too many outside references: streaming kernel
    const int64_t smem = 8LL * stats[1] + 4LL * (stats[0] + 1) + 8LL * stats[0] + 8LL * stats[2];
    if (smem > smem_optin || smem * per_sm > smem_sm - 2048 * per_sm) continue;
    PCK(launch_scan(p.hcount, p.hoff, B, p.scan_tmp, st));
    int32_t htot = 0;
    PCK(cudaMemcpyAsync(&htot, p.hoff + B, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    PCK(grow(&p.halo, &p.halo_cap, htot > 0 ? htot : 1));
    plan_map_kernel<<<B, 512, 0, st>>>(p.irp, p.iec, p.part, p.tmp, p.hoff, p.halo, p.lec);
    count_launch();
    PCK(cudaGetLastError());
    p.B = B;
    p.threads = threads;
    p.maxO = stats[0];
    p.maxE = stats[1];
    p.maxH = stats[2];
    p.smem = (size_t)smem;
    p.halo_total = htot;
    p.valid = true;
    return cudaSuccess;
  }
  return cudaSuccess;  // does not fit: streaming kernel
}

template <int G>
static cudaError_t launch_tiled_g(GdpPlan& p, int32_t F, int32_t shift, int64_t max_sweeps,
                                  GdpCtl* ctl, long long* trace_b2, unsigned long long* trace_ch,
                                  int64_t trace_cap, long long budget, cudaStream_t st) {
  PCK(cudaFuncSetAttribute(gdp_tiled_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  int per_sm = 0;
  PCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gdp_tiled_kernel<G>, p.threads, p.smem));
  int dev = 0, sms = 0;
  PCK(cudaGetDevice(&dev));
  PCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if ((long long)per_sm * sms < p.B) return cudaErrorCooperativeLaunchTooLarge;
  long long ms = max_sweeps, tc = trace_cap;
  int32_t* l0 = p.ilam[0];
  int32_t* l1 = p.ilam[1];
  void* args[] = {(void*)&p.irp, (void*)&p.lec, (void*)&p.part, (void*)&p.hoff, (void*)&p.halo,
                  (void*)&l0, (void*)&l1, (void*)&F, (void*)&shift, (void*)&ms, (void*)&ctl,
                  (void*)&trace_b2, (void*)&trace_ch, (void*)&tc, (void*)&budget, (void*)&p.maxE,
                  (void*)&p.maxO, (void*)&p.maxH};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)gdp_tiled_kernel<G>, dim3(p.B),
                                              dim3(p.threads), args, p.smem, st);
  count_launch();
  return e;
}

cudaError_t launch_gdp_tiled(GdpPlan& p, const int32_t* lam_in, int32_t F, int32_t shift,
                             int64_t max_sweeps, GdpCtl* ctl, long long* trace_b2,
                             unsigned long long* trace_ch, int64_t trace_cap, long long budget,
                             cudaStream_t st) {
  PCK(gather_perm(lam_in, p.perm, p.n, p.ilam[0], st));
  return launch_tiled_g<4>(p, F, shift, max_sweeps, ctl, trace_b2, trace_ch, trace_cap, budget, st);
}

cudaError_t plan_scatter_lambda(const GdpPlan& p, int which, int32_t* lam_out, cudaStream_t st) {
  return scatter_perm(p.ilam[which], p.perm, p.n, lam_out, st);
}

}  // namespace f2m
