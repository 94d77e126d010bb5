// Batched GDP on thread-block clusters: one cluster per instance, the
// instance's rows and lambda resident in the cluster's shared memory.
//
// The instances of a batch never interact, so a sweep needs a barrier only
// among the CTAs that hold one instance.  An instance of n nodes goes to a
// cluster of C = 1, 2, 4, 8 or 16 CTAs (the smallest that holds it): CTA r
// owns the internal (Morton-renumbered) nodes [node0 + r*per, node0 + (r+1)*per)
// with per = ceil(n / C), their rows as {packed column, cost * 2^F} and two
// lambda buffers.  A column is packed as (owner rank << 16 | local index), so
// a neighbour's lambda is read from the owner's shared memory, through the
// distributed shared memory window when the owner is another CTA of the
// cluster.  One sweep (Section 4, Eq. 9 and Eq. 10; Section 5.1, Jacobi):
// every CTA updates its own nodes from lambda ring slot t % 3 into the next,
// writes its changed count to slot t & 1, and the cluster meets at the
// hardware cluster barrier (the cluster's __syncthreads).  While sweep t + 1
// runs, every CTA reads the C counts of sweep t; the cluster stops after the
// first sweep that changed nothing (lambda is then the same in both slots),
// on overflow (the sweep's input, kept by the ring of three, is the result) or
// at max_sweeps.  The stop decision comes from the same counts in every CTA,
// so all CTAs take the same number of barriers.  The arithmetic is that of
// the other GDP kernels, so every instance's sweeps are bit for bit those of
// its own solve.
#include <climits>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared::cluster address of the same location in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ int ld_cluster(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_hw() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace

__global__ void __launch_bounds__(1024, 1)
gdp_cluster_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ pk,
                   const ClusterInst* __restrict__ insts, int32_t* ilam, int32_t shift,
                   long long max_sweeps, ClusterOut* out, int32_t emax, int32_t nmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  int2* s_ent = reinterpret_cast<int2*>(smem);              // own rows {packed col, cost << F}
  int* s_rp = reinterpret_cast<int*>(s_ent + emax);          // own row offsets [nmax + 1]
  int* s_lam = s_rp + nmax + 1;                              // lambda, a ring of three [3][nmax]
  __shared__ int s_cnt[2];                                   // changed count per sweep parity
  __shared__ int s_ovf[2];
  __shared__ int s_prev;                                     // verdict on the previous sweep
  __shared__ int s_red[32];
  __shared__ int s_oflag[32];

  uint32_t ncta;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
  const uint32_t rank = cluster_rank();
  const ClusterInst in = insts[blockIdx.x / ncta];
  const int tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int a = in.node0 + (int)rank * in.per;
  int b = a + in.per;
  if (b > in.node0 + in.n) b = in.node0 + in.n;
  const int own = b > a ? b - a : 0;  // a CTA past the instance's end owns nothing
  const int e0 = own > 0 ? irp[a] : 0;
  const int ne = own > 0 ? irp[b] - e0 : 0;

  for (int e = tid; e < ne; e += T) s_ent[e] = pk[e0 + e];
  for (int i = tid; i <= own; i += T) s_rp[i] = (own > 0 ? irp[a + i] : 0) - e0;
  for (int i = tid; i < own; i += T) s_lam[i] = ilam[a + i];
  cluster_sync_hw();  // every CTA started and initialised

  const uint32_t lam_base = smem_addr(s_lam);
  // verdict on sweep t from the cluster's counts: 2 overflow, 1 nothing changed
  auto verdict = [&](long long t) {
    if (warp == 0) {
      const int p = (int)(t & 1);
      int c = 0, o = 0;
      if (lane < (int)ncta) {
        c = ld_cluster(map_rank(smem_addr(&s_cnt[p]), (uint32_t)lane));
        o = ld_cluster(map_rank(smem_addr(&s_ovf[p]), (uint32_t)lane));
      }
      c = __reduce_add_sync(0xffffffffu, c);
      o = __reduce_or_sync(0xffffffffu, o);
      if (lane == 0) s_prev = o ? 2 : (c == 0 ? 1 : 0);
    }
  };
  long long done = -1;
  int status = 0, fixed = 0, res = 0;
  for (long long t = 0; t < max_sweeps; ++t) {
    // sweep t reads ring slot t % 3 and writes (t + 1) % 3, so the input of
    // sweep t - 1 survives sweep t; the verdict on sweep t - 1 (its counts are
    // complete since the last barrier) is taken while sweep t runs
    const int pin = (int)(t % 3), pout = (int)((t + 1) % 3);
    const int* lin = s_lam + pin * nmax;
    int* lout = s_lam + pout * nmax;
    const uint32_t rin = lam_base + (uint32_t)(pin * nmax) * 4u;
    if (t >= 1) verdict(t - 1);
    int ch = 0, ovf = 0;
    for (int v = tid; v < own; v += T) {
      const int lv = lin[v];
      int x0 = INT_MAX, x1 = INT_MAX, x2 = INT_MAX;
      for (int e = s_rp[v]; e < s_rp[v + 1]; ++e) {
        const int2 q = s_ent[e];
        const uint32_t r = (uint32_t)q.x >> 16;
        const int l = q.x & 0xFFFF;
        const int lu = r == rank ? lin[l] : ld_cluster(map_rank(rin + 4u * (uint32_t)l, r));
        top3_insert_minmax(q.y - lv - lu, x0, x1, x2);  // Eq. 9
      }
      const long long d = gdp_step(x1, x2, shift);  // Eq. 10, truncated toward 0
      const long long nl = (long long)lv + d;
      ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
      ch += (d != 0);
      lout[v] = (int32_t)nl;
    }
    ch = __reduce_add_sync(0xffffffffu, ch);
    ovf = __reduce_or_sync(0xffffffffu, ovf);
    if (lane == 0) { s_red[warp] = ch; s_oflag[warp] = ovf; }
    __syncthreads();
    if (tid == 0) {
      int c = 0, o = 0;
      for (int w = 0; w < nwarps; ++w) { c += s_red[w]; o |= s_oflag[w]; }
      s_cnt[t & 1] = c;
      s_ovf[t & 1] = o;
    }
    if (t >= 1 && s_prev != 0) {  // the same verdict in every CTA: stop together
      done = t;                   // sweeps run up to the decisive one, t - 1
      if (s_prev == 2) {          // overflow: lambda stays at the input of sweep t - 1
        status |= kGdpOverflow;
        res = (int)((t - 1) % 3);
      } else {                    // sweep t - 1 changed nothing
        fixed = 1;
        res = pin;
      }
      break;
    }
    cluster_sync_hw();  // sweep t complete everywhere
  }
  if (done < 0) {
    done = max_sweeps > 0 ? max_sweeps : 0;
    res = (int)(done % 3);
    if (done > 0) {
      verdict(done - 1);
      __syncthreads();
      if (s_prev == 2) {
        status |= kGdpOverflow;
        res = (int)((done - 1) % 3);
      } else if (s_prev == 1) {
        fixed = 1;
      }
    }
  }
  for (int i = tid; i < own; i += T) ilam[a + i] = s_lam[res * nmax + i];
  if (rank == 0 && tid == 0) out[in.seg] = ClusterOut{done, status, fixed};
  cluster_sync_hw();  // no CTA leaves while another may read its shared memory
}

// pk[e] for every entry of the listed instances: {owner rank << 16 | local, cost << F}
__global__ void cluster_pack_kernel(const int32_t* __restrict__ irp, const int2* __restrict__ iec,
                                    const ClusterInst* __restrict__ insts, int32_t ninst, int32_t F,
                                    int2* __restrict__ pk) {
  const ClusterInst in = insts[blockIdx.x];
  for (int i = threadIdx.x; i < in.n; i += blockDim.x) {
    const int v = in.node0 + i;
    for (int e = irp[v]; e < irp[v + 1]; ++e) {
      const int2 q = iec[e];
      const int u = q.x - in.node0;  // same instance
      const int r = u / in.per, l = u - r * in.per;
      pk[e] = make_int2((r << 16) | l, q.y << F);
    }
  }
}

cudaError_t cluster_pack(const int32_t* irp, const int2* iec, const ClusterInst* d_insts, int32_t ninst,
                         int32_t F, int2* pk, cudaStream_t st) {
  if (ninst <= 0) return cudaSuccess;
  cluster_pack_kernel<<<ninst, 256, 0, st>>>(irp, iec, d_insts, ninst, F, pk);
  count_launch();
  return cudaGetLastError();
}

size_t cluster_smem(int32_t emax, int32_t nmax) {
  return (size_t)emax * 8 + (size_t)(nmax + 1) * 4 + (size_t)3 * nmax * 4;
}

cudaError_t launch_gdp_cluster(int32_t C, int32_t threads, const int32_t* irp, const int2* pk,
                               const ClusterInst* d_insts, int32_t ninst, int32_t* ilam,
                               int32_t shift, int64_t max_sweeps, ClusterOut* out,
                               int32_t emax, int32_t nmax, cudaStream_t st) {
  if (ninst <= 0) return cudaSuccess;
  const size_t smem = cluster_smem(emax, nmax);
  cudaError_t e = cudaFuncSetAttribute(gdp_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && C > 8)
    e = cudaFuncSetAttribute(gdp_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ninst * C));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  long long ms = max_sweeps;
  e = cudaLaunchKernelEx(&cfg, gdp_cluster_kernel, irp, pk, d_insts, ilam, shift, ms, out, emax, nmax);
  count_launch();
  return e;
}

int32_t cluster_max_smem_ok(int32_t C, int32_t threads, int32_t emax, int32_t nmax) {
  // 1 if a cluster of C CTAs with this shared memory can be resident at all
  const size_t smem = cluster_smem(emax, nmax);
  if (cudaFuncSetAttribute(gdp_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (C > 8 && cudaFuncSetAttribute(gdp_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, gdp_cluster_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nclusters;
}

}  // namespace f2m
