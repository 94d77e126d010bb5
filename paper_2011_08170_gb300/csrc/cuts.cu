// Subtour-elimination cuts: GDP over node and cut duals.
//
// The paper's Discussion names the F2M LP plus subtour elimination constraints
// as the next relaxation for the method.  The LP:
//   minimise c x  subject to  x(delta(v)) = 2 for every node v      (Section 4)
//                             x(delta(S)) >= 2 for every cut S of a family
//                             0 <= x <= 1,
// Section 2's LP3 with equalities (1) and inequalities (2).  Every constraint
// has binary coefficients and right side 2 (Eq. 8), so Section 3's gradient
// applies to each: the 2nd and 3rd smallest modified values over its support.
// Inequality duals stay >= 0 (Eq. 5).  The modified objective (Eq. 4) of an
// edge uv is
//   z_uv = c_uv 2^F - lambda_u - lambda_v - sum of mu_S over the cuts S that
//          hold exactly one of u, v.
// One Jacobi sweep (Section 5.1's parallel update, extended to the cut duals)
// reads only the previous lambda and mu:
//   lambda_v += trunc((z(2) + z(3)) / 2^shift) over delta(v),
//   mu_S = max(0, mu_S + trunc((z(2) + z(3)) / 2^(shift + 2))) over delta(S),
// the cut step a quarter of the node step: an edge's z moves with both end
// duals and with up to two cut duals per layer at once, and nested cuts of
// different layers move nearly the same edges (a full node-sized step made
// the duals diverge after a few layers);
//   bound2 = 4 sum lambda + 4 sum mu + sum over directed entries of min(0, z).
//
// Cut family: up to kMaxCutLayers layers; layer l labels every node with -1
// (no cut of the layer) or a cut index s in [0, ncuts_l); the nodes labelled s
// form the cut set.  Cuts of one layer are disjoint.  Separation makes one
// layer from the connected components of the support of x.
//
// Device layout (caller node order, like the streaming GDP kernel):
//   comp [L][n] int32 labels; mu [2][M] int32 (Jacobi double buffer);
//   mask [nnz] uint8 (bit l: the entry's two ends differ in layer l's label);
//   cut lists: cut_ptr [M+1], items {row u, entry e} for every directed entry
//   whose row lies in the cut and whose column does not (each crossing edge
//   once per cut).
// Kernel: one persistent cooperative launch per phase.  G = 4 lanes per node
// stream its row (cut terms only on entries whose mask is set), then one warp
// per cut streams its list (a whole block for a cut with 128 or more entries,
// its warps' top-3s merged in shared memory); both from the same input, one
// device-wide barrier per sweep.  z is computed in 64 bits (several duals per
// edge).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/f2m.h"
#include "ctx_internal.h"
#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

struct CutArgs {
  const int32_t* comp;  // [L][n]
  int32_t n, L;
  int32_t off[kMaxCutLayers + 1];  // first cut index of each layer
};

struct CutState {
  int32_t L = 0;
  std::vector<int32_t> ncuts;  // per layer
  std::vector<int32_t> off;    // [L + 1]
  int64_t M = 0;               // cuts in all layers
  int32_t* d_comp = nullptr;   // [kMaxCutLayers][n]
  int32_t* d_mu[2] = {nullptr, nullptr};
  int64_t mu_cap = 0;
  int cur = 0;                 // d_mu[cur] holds mu
  uint8_t* d_mask = nullptr;
  int64_t mask_cap = 0;
  int32_t* d_cnt = nullptr;    // per cut: count, then fill cursor
  int32_t* d_ptr = nullptr;    // [M + 1]
  int32_t* d_scan = nullptr;   // scan scratch
  int64_t ptr_cap = 0;
  int2* d_items = nullptr;
  int64_t item_cap = 0;
  int64_t items = 0;
  int32_t* d_lflag = nullptr;  // [ptr_cap] long-cut flags
  int32_t* d_lpos = nullptr;   // [ptr_cap] their exclusive scan
  int32_t* d_long = nullptr;   // [ptr_cap] the cuts a block takes
  int32_t nlong = 0;
  int64_t built_version = -1;  // graph version the mask and lists were built for
  int32_t built_L = -1;
  // separation and pricing scratch
  int32_t* d_lab = nullptr;    // [n] component label (smallest node)
  int32_t* d_cross = nullptr;  // [n] crossing entries per root
  int32_t* d_flag = nullptr;   // [n + 1] flags, then ranks
  int32_t* d_rank = nullptr;   // [n + 1]
  int32_t* d_small = nullptr;  // [4] small device counters
  int32_t* d_lamp = nullptr;   // [n] lambda + the duals of the cuts holding the node
  int32_t* d_keep = nullptr;   // [pair_cap + 1]
  int32_t* d_kpos = nullptr;   // [pair_cap + 1]
  int2* d_pairs2 = nullptr;
  int64_t pair_cap = 0;
  int32_t* d_pscan = nullptr;
  int64_t pscan_cap = 0;
};

void cut_state_free(CutState* s) {
  if (!s) return;
  dfree(s->d_comp); dfree(s->d_mu[0]); dfree(s->d_mu[1]); dfree(s->d_mask); dfree(s->d_cnt);
  dfree(s->d_ptr); dfree(s->d_scan); dfree(s->d_items); dfree(s->d_lab); dfree(s->d_cross);
  dfree(s->d_flag); dfree(s->d_rank); dfree(s->d_small); dfree(s->d_lamp); dfree(s->d_keep);
  dfree(s->d_kpos); dfree(s->d_pairs2); dfree(s->d_pscan); dfree(s->d_lflag); dfree(s->d_lpos);
  dfree(s->d_long);
  delete s;
}

int64_t cut_count(const f2m_ctx* c) { return c->cuts ? c->cuts->M : 0; }

namespace {

constexpr long long kInfZ = LLONG_MAX / 4;
constexpr int kLongCut = 128;  // crossing entries from which a block, not a warp, takes a cut

__device__ __forceinline__ void top3_ins_ll(long long z, long long& a, long long& b, long long& c) {
  if (z < c) {
    if (z < b) {
      c = b;
      if (z < a) { b = a; a = z; } else { b = z; }
    } else {
      c = z;
    }
  }
}

__device__ __forceinline__ long long step_ll(long long z2, long long z3, int shift) {
  const long long s = z2 + z3;
  return s >= 0 ? (s >> shift) : -((-s) >> shift);  // truncation toward zero
}

__device__ __forceinline__ long long ld_cg_i(const int32_t* p) { return (long long)__ldcg(p); }

// sum of the duals of the cuts that entry (u, v) crosses; bit l of m set when
// the ends differ in layer l's label
__device__ __forceinline__ long long cut_term(const CutArgs& a, const int32_t* mu, unsigned m, int u, int v) {
  long long t = 0;
  for (int l = 0; l < a.L; ++l) {
    if (!((m >> l) & 1u)) continue;
    const int cu = __ldg(a.comp + (long long)l * a.n + u), cv = __ldg(a.comp + (long long)l * a.n + v);
    if (cu >= 0) t += ld_cg_i(mu + a.off[l] + cu);
    if (cv >= 0) t += ld_cg_i(mu + a.off[l] + cv);
  }
  return t;
}

__device__ __forceinline__ long long entry_z(const CutArgs& a, const int32_t* lam, const int32_t* mu,
                                             unsigned m, int u, int2 q, int F) {
  long long z = ((long long)q.y << F) - ld_cg_i(lam + u) - ld_cg_i(lam + q.x);
  if (m) z -= cut_term(a, mu, m, u, q.x);
  return z;
}

// mask[e] for every directed entry
__global__ void cut_mask_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec, CutArgs a,
                                uint8_t* __restrict__ mask) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < a.n;
       v += (long long)gridDim.x * blockDim.x) {
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      const int w = ec[e].x;
      unsigned m = 0;
      for (int l = 0; l < a.L; ++l)
        if (a.comp[(long long)l * a.n + v] != a.comp[(long long)l * a.n + w]) m |= 1u << l;
      mask[e] = (uint8_t)m;
    }
  }
}

// per cut: crossing entries whose row lies in the cut (count, or fill at the
// cursor); a label outside [-1, ncuts) flags the layer as invalid
template <bool FILL>
__global__ void cut_list_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                const uint8_t* __restrict__ mask, CutArgs a, int32_t* cnt,
                                const int32_t* __restrict__ ptr, int2* items) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < a.n;
       v += (long long)gridDim.x * blockDim.x) {
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      const unsigned m = mask[e];
      if (!m) continue;
      for (int l = 0; l < a.L; ++l) {
        if (!((m >> l) & 1u)) continue;
        const int s = a.comp[(long long)l * a.n + v];
        if (s < 0) continue;
        const int id = a.off[l] + s;
        const int k = atomicAdd(cnt + id, 1);
        if (FILL) items[ptr[id] + k] = make_int2((int)v, e);
      }
    }
  }
}

// 1 for a cut whose list holds at least kLongCut entries
__global__ void cut_long_flag_kernel(const int32_t* __restrict__ cnt, int32_t M, int32_t* flag) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < M;
       s += (long long)gridDim.x * blockDim.x)
    flag[s] = cnt[s] >= kLongCut;
}

__global__ void cut_long_list_kernel(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                     int32_t M, int32_t* out) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < M;
       s += (long long)gridDim.x * blockDim.x)
    if (flag[s]) out[pos[s]] = (int32_t)s;
}

// labels of layer l in [-1, ncuts): else flag
__global__ void cut_label_check_kernel(const int32_t* __restrict__ comp, int32_t n, int32_t ncuts,
                                       int32_t* flag) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int s = comp[v];
    if (s < -1 || s >= ncuts) atomicMin(flag, (int)v);
  }
}

// cuts with fewer than 3 crossing edges: smallest such cut index into flag
__global__ void cut_short_kernel(const int32_t* __restrict__ cnt, int32_t M, int32_t* flag) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < M;
       s += (long long)gridDim.x * blockDim.x)
    if (cnt[s] < 3) atomicMin(flag, (int)s);
}

template <int G>
__global__ void __launch_bounds__(512)
cut_gdp_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec, const uint8_t* __restrict__ mask,
               const __grid_constant__ CutArgs ca, const int32_t* __restrict__ cut_ptr, const int2* __restrict__ items,
               int32_t M, const int32_t* __restrict__ long_cuts, int32_t nlong,
               int32_t* lam0, int32_t* lam1, int32_t* mu0, int32_t* mu1, int32_t F, int32_t shift,
               long long max_sweeps, GdpCtl* ctl, long long* trace_b2, unsigned long long* trace_ch,
               long long trace_cap, long long budget) {
  __shared__ long long s_b2[32];
  __shared__ unsigned s_ch[32];
  __shared__ int s_ovf[32];
  __shared__ int s_stop;
  __shared__ long long s_t3[32 * 3];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int sub = lane & (G - 1);
  const unsigned gmask = (G >= 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const long long per_block = blockDim.x / G;
  const long long gid = (long long)blockIdx.x * per_block + tid / G;
  const long long ngroups = (long long)gridDim.x * per_block;
  const int nwarps = blockDim.x >> 5;
  const long long gwarp = (long long)blockIdx.x * nwarps + warp;
  const long long twarps = (long long)gridDim.x * nwarps;
  const int n = ca.n;

  for (long long t = 0; t < max_sweeps; ++t) {
    const int32_t* lin = (t & 1) ? lam1 : lam0;
    int32_t* lout = (t & 1) ? lam0 : lam1;
    const int32_t* min_ = (t & 1) ? mu1 : mu0;
    int32_t* mout = (t & 1) ? mu0 : mu1;
    long long b2 = 0;
    unsigned ch = 0;
    int ovf = 0;
    // node duals: Section 3's gradient over delta(v)
    for (long long v = gid; v < n; v += ngroups) {
      const int beg = __ldg(rp + v), end = __ldg(rp + v + 1);
      long long a = kInfZ, b = kInfZ, c = kInfZ;
      for (int e = beg + sub; e < end; e += G) {
        const long long z = entry_z(ca, lin, min_, __ldg(mask + e), (int)v, __ldg(ec + e), F);
        if (z < 0) b2 += z;
        top3_ins_ll(z, a, b, c);
      }
      for (int o = 1; o < G; o <<= 1) {
        const long long a1 = __shfl_xor_sync(gmask, a, o), b1 = __shfl_xor_sync(gmask, b, o),
                        c1 = __shfl_xor_sync(gmask, c, o);
        top3_ins_ll(a1, a, b, c);
        top3_ins_ll(b1, a, b, c);
        top3_ins_ll(c1, a, b, c);
      }
      if (sub == 0) {
        const long long lv = ld_cg_i(lin + v);
        const long long d = step_ll(b, c, shift);
        const long long nl = lv + d;
        ovf |= (nl >= kLamLimit || nl <= -kLamLimit);
        lout[v] = (int32_t)nl;
        ch += (d != 0);
        b2 += 4 * lv;
      }
    }
    // cut duals: Section 3's gradient over delta(S), projected onto mu >= 0.
    // A cut with a long list is taken by a whole block (its warps' top-3s
    // merged in shared memory), the others by one warp each.
    auto cut_update = [&](long long s, long long a, long long b, long long c) {
      const long long m = ld_cg_i(min_ + s);
      long long nm = m + step_ll(b, c, shift + 2);
      if (nm < 0) nm = 0;
      ovf |= (nm >= kLamLimit);
      mout[s] = (int32_t)nm;
      ch += (nm != m);
      b2 += 4 * m;
    };
    for (long long q = blockIdx.x; q < nlong; q += gridDim.x) {
      const int s = __ldg(long_cuts + q);
      const int p0 = __ldg(cut_ptr + s), p1 = __ldg(cut_ptr + s + 1);
      long long a = kInfZ, b = kInfZ, c = kInfZ;
      for (int k = p0 + tid; k < p1; k += blockDim.x) {
        const int2 it = __ldg(items + k);
        top3_ins_ll(entry_z(ca, lin, min_, __ldg(mask + it.y), it.x, __ldg(ec + it.y), F), a, b, c);
      }
      for (int o = 1; o < 32; o <<= 1) {
        const long long a1 = __shfl_xor_sync(0xffffffffu, a, o), b1 = __shfl_xor_sync(0xffffffffu, b, o),
                        c1 = __shfl_xor_sync(0xffffffffu, c, o);
        top3_ins_ll(a1, a, b, c);
        top3_ins_ll(b1, a, b, c);
        top3_ins_ll(c1, a, b, c);
      }
      if (lane == 0) { s_t3[3 * warp] = a; s_t3[3 * warp + 1] = b; s_t3[3 * warp + 2] = c; }
      __syncthreads();
      if (warp == 0) {
        a = lane < nwarps ? s_t3[3 * lane] : kInfZ;
        b = lane < nwarps ? s_t3[3 * lane + 1] : kInfZ;
        c = lane < nwarps ? s_t3[3 * lane + 2] : kInfZ;
        for (int o = 1; o < 32; o <<= 1) {
          const long long a1 = __shfl_xor_sync(0xffffffffu, a, o), b1 = __shfl_xor_sync(0xffffffffu, b, o),
                          c1 = __shfl_xor_sync(0xffffffffu, c, o);
          top3_ins_ll(a1, a, b, c);
          top3_ins_ll(b1, a, b, c);
          top3_ins_ll(c1, a, b, c);
        }
        if (lane == 0) cut_update(s, a, b, c);
      }
      __syncthreads();
    }
    for (long long s = gwarp; s < M; s += twarps) {
      const int p0 = __ldg(cut_ptr + s), p1 = __ldg(cut_ptr + s + 1);
      if (p1 - p0 >= kLongCut) continue;  // a block's
      long long a = kInfZ, b = kInfZ, c = kInfZ;
      for (int k = p0 + lane; k < p1; k += 32) {
        const int2 it = __ldg(items + k);
        top3_ins_ll(entry_z(ca, lin, min_, __ldg(mask + it.y), it.x, __ldg(ec + it.y), F), a, b, c);
      }
      for (int o = 1; o < 32; o <<= 1) {
        const long long a1 = __shfl_xor_sync(0xffffffffu, a, o), b1 = __shfl_xor_sync(0xffffffffu, b, o),
                        c1 = __shfl_xor_sync(0xffffffffu, c, o);
        top3_ins_ll(a1, a, b, c);
        top3_ins_ll(b1, a, b, c);
        top3_ins_ll(c1, a, b, c);
      }
      if (lane == 0) cut_update(s, a, b, c);
    }
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
        const int sl = (int)(t % 3);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->slot_b2[sl]), (unsigned long long)x);
        if (y) atomicAdd(&ctl->slot_ch[sl], (unsigned long long)y);
        if (o) atomicOr(&ctl->status, kGdpOverflow);
      }
    }
    const bool ok = grid_barrier(&ctl->bar_count, &ctl->bar_gen, gridDim.x, budget);
    if (tid == 0) {
      if (!ok) atomicOr(&ctl->status, kGdpTimeout);
      volatile GdpCtl* vc = ctl;
      const int sl = (int)(t % 3);
      const unsigned long long chg = vc->slot_ch[sl];
      const int st = vc->status;
      if (blockIdx.x == 0) {
        if (t < trace_cap) {
          trace_b2[t] = vc->slot_b2[sl];
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

// bound2 at (lam, mu) with fb bits, and (x2 != NULL) rule (7) with the cut terms
__global__ void cut_bound_extract_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                         const uint8_t* __restrict__ mask, CutArgs ca,
                                         const int32_t* __restrict__ lam, const int32_t* __restrict__ mu,
                                         int32_t M, int32_t fb, uint8_t* x2, long long* b2_out,
                                         unsigned long long* bad) {
  long long b2 = 0;
  unsigned nb = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < ca.n; v += stride) {
    int s = 0;
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      const long long z = entry_z(ca, lam, mu, mask[e], (int)v, ec[e], fb);
      if (z < 0) b2 += z;
      const int x = z < 0 ? 2 : (z == 0 ? 1 : 0);
      if (x2) x2[e] = (uint8_t)x;
      s += x;
    }
    b2 += 4LL * lam[v];
    nb += (s != 4);
  }
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < M; q += stride) b2 += 4LL * mu[q];
  b2 = warp_sum_ll(b2);
  nb = warp_sum_u(nb);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(b2_out), (unsigned long long)b2);
    if (nb) atomicAdd(bad, (unsigned long long)nb);
  }
}

// ---- separation: connected components of the support {e : x2_e > 0} -------

__global__ void cc_init_kernel(int32_t* lab, int32_t n) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    lab[v] = (int32_t)v;
}

// hook the larger of two roots under the smaller along every support entry
__global__ void cc_hook_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                               const uint8_t* __restrict__ x2, int32_t n, int32_t* lab, int32_t* changed) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      if (!x2[e]) continue;
      const int a = __ldcg(lab + v), b = __ldcg(lab + ec[e].x);
      if (a == b) continue;
      const int hi = a > b ? a : b, lo = a > b ? b : a;
      if (atomicMin(lab + hi, lo) > lo) *changed = 1;
    }
  }
}

// pointer jumping to the root
__global__ void cc_compress_kernel(int32_t* lab, int32_t n, int32_t* changed) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    int r = __ldcg(lab + v);
    int rr = __ldcg(lab + r);
    if (rr == r) continue;
    while (rr != r) {
      r = rr;
      rr = __ldcg(lab + r);
    }
    lab[v] = r;
    *changed = 1;
  }
}

// crossing candidate entries per component (by root), and the root flags
__global__ void cc_cross_kernel(const int32_t* __restrict__ rp, const int2* __restrict__ ec,
                                const int32_t* __restrict__ lab, int32_t n, int32_t* cross, int32_t* root) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int a = lab[v];
    int k = 0;
    for (int e = rp[v]; e < rp[v + 1]; ++e) k += (lab[ec[e].x] != a);
    if (k) atomicAdd(cross + a, k);
    root[v] = (a == (int)v);
  }
}

// which components become cuts: all if m >= 3, the one without node 0 if m = 2;
// only those with at least 3 crossing candidate edges
__global__ void cc_keep_kernel(const int32_t* __restrict__ lab, const int32_t* __restrict__ cross,
                               int32_t n, int32_t m, int32_t* keep) {
  const int r0 = lab[0];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const bool is_root = lab[v] == (int)v;
    const bool take = m >= 3 || (m == 2 && (int)v != r0);
    keep[v] = (is_root && take && cross[v] >= 3) ? 1 : 0;
  }
}

__global__ void cc_label_kernel(const int32_t* __restrict__ lab, const int32_t* __restrict__ keep,
                                const int32_t* __restrict__ rank, int32_t n, int32_t* comp) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int r = lab[v];
    comp[v] = keep[r] ? rank[r] : -1;
  }
}

// ---- pricing with cuts -----------------------------------------------------

// lamp_v = lambda_v + the duals of the cuts holding v: z_uv >= c 2^fb - lamp_u -
// lamp_v, so the plain scan with lamp finds a superset of the pairs
__global__ void cut_lamp_kernel(CutArgs ca, const int32_t* __restrict__ lam, const int32_t* __restrict__ mu,
                                int32_t* lamp, int32_t* overflow) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < ca.n;
       v += (long long)gridDim.x * blockDim.x) {
    long long x = lam[v];
    for (int l = 0; l < ca.L; ++l) {
      const int s = ca.comp[(long long)l * ca.n + v];
      if (s >= 0) x += mu[ca.off[l] + s];
    }
    if (x >= INT_MAX || x <= INT_MIN) {
      atomicOr(overflow, 1);
      x = 0;
    }
    lamp[v] = (int32_t)x;
  }
}

// exact z with the cut terms for every pair of the superset: keep flags
__global__ void cut_pair_keep_kernel(const int2* __restrict__ pairs, long long np, const int2* __restrict__ xy,
                                     CutArgs ca, const int32_t* __restrict__ lam, const int32_t* __restrict__ mu,
                                     int32_t fb, int32_t* keep) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < np;
       k += (long long)gridDim.x * blockDim.x) {
    const int2 p = pairs[k];
    long long t = 0;
    for (int l = 0; l < ca.L; ++l) {
      const int cu = ca.comp[(long long)l * ca.n + p.x], cv = ca.comp[(long long)l * ca.n + p.y];
      if (cu != cv) {
        if (cu >= 0) t += mu[ca.off[l] + cu];
        if (cv >= 0) t += mu[ca.off[l] + cv];
      }
    }
    const long long z = ((long long)exact_cost(xy[p.x], xy[p.y]) << fb) - lam[p.x] - lam[p.y] - t;
    keep[k] = z < 0;
  }
}

__global__ void cut_pair_compact_kernel(const int2* __restrict__ pairs, long long np,
                                        const int32_t* __restrict__ keep, const int32_t* __restrict__ pos,
                                        int2* out) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < np;
       k += (long long)gridDim.x * blockDim.x)
    if (keep[k]) out[pos[k]] = pairs[k];
}

int grid_of(long long items, int threads) {
  long long b = (items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

CutArgs cut_args(const f2m_ctx* c) {
  CutArgs a{};
  a.comp = c->cuts->d_comp;
  a.n = c->n;
  a.L = c->cuts->L;
  for (int l = 0; l <= c->cuts->L; ++l) a.off[l] = c->cuts->off[l];
  return a;
}

template <typename T>
cudaError_t grow(T** p, int64_t* cap, int64_t need) {
  if (need <= *cap) return cudaSuccess;
  dfree(*p);
  *cap = need + need / 4 + 16;
  return dalloc(p, *cap);
}

}  // namespace

// Mask and cut lists for the graph held now (rebuilt after a merge or a new layer).
f2m_status cut_lists(f2m_ctx* c) {
  CutState* S = c->cuts;
  if (S->built_version == c->plan.version && S->built_L == S->L) return F2M_OK;
  const CutArgs a = cut_args(c);
  CK(c, grow(&S->d_mask, &S->mask_cap, c->nnz));
  cut_mask_kernel<<<grid_of(c->n, 256), 256, 0, c->st>>>(c->d_rp, c->d_ec, a, S->d_mask);
  count_launch();
  if (S->ptr_cap < S->M + 1) {
    dfree(S->d_cnt);
    dfree(S->d_ptr);
    dfree(S->d_scan);
    dfree(S->d_lflag);
    dfree(S->d_lpos);
    dfree(S->d_long);
    S->ptr_cap = S->M + 1 + 1024;
    CK(c, dalloc(&S->d_cnt, S->ptr_cap));
    CK(c, dalloc(&S->d_ptr, S->ptr_cap));
    CK(c, dalloc(&S->d_scan, (int64_t)scan_scratch_ints((int32_t)S->ptr_cap)));
    CK(c, dalloc(&S->d_lflag, S->ptr_cap));
    CK(c, dalloc(&S->d_lpos, S->ptr_cap));
    CK(c, dalloc(&S->d_long, S->ptr_cap));
  }
  CK(c, cudaMemsetAsync(S->d_cnt, 0, sizeof(int32_t) * (S->M + 1), c->st));
  cut_list_kernel<false><<<grid_of(c->n, 256), 256, 0, c->st>>>(c->d_rp, c->d_ec, S->d_mask, a, S->d_cnt,
                                                                  nullptr, nullptr);
  count_launch();
  CK(c, launch_scan(S->d_cnt, S->d_ptr, (int32_t)S->M, S->d_scan, c->st));
  int32_t total = 0;
  CK(c, cudaMemcpyAsync(&total, S->d_ptr + S->M, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  CK(c, grow(&S->d_items, &S->item_cap, (int64_t)total));
  CK(c, cudaMemsetAsync(S->d_cnt, 0, sizeof(int32_t) * (S->M + 1), c->st));
  cut_list_kernel<true><<<grid_of(c->n, 256), 256, 0, c->st>>>(c->d_rp, c->d_ec, S->d_mask, a, S->d_cnt,
                                                                 S->d_ptr, S->d_items);
  count_launch();
  CK(c, cudaGetLastError());
  // the cuts with long lists, in index order
  cut_long_flag_kernel<<<grid_of(S->M, 256), 256, 0, c->st>>>(S->d_cnt, (int32_t)S->M, S->d_lflag);
  count_launch();
  CK(c, launch_scan(S->d_lflag, S->d_lpos, (int32_t)S->M, S->d_scan, c->st));
  cut_long_list_kernel<<<grid_of(S->M, 256), 256, 0, c->st>>>(S->d_lflag, S->d_lpos, (int32_t)S->M, S->d_long);
  count_launch();
  int32_t nlong = 0;
  CK(c, cudaMemcpyAsync(&nlong, S->d_lpos + S->M, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  S->nlong = nlong;
  S->items = total;
  S->built_version = c->plan.version;
  S->built_L = S->L;
  return F2M_OK;
}

f2m_status cut_gdp_phase(f2m_ctx* c, int64_t max_sweeps, int64_t* sweeps, long long* tb,
                         unsigned long long* tc, int64_t tcap, double* ms) {
  CutState* S = c->cuts;
  c->lam_version += 1;
  f2m_status s = cut_lists(c);
  if (s != F2M_OK) return s;
  const CutArgs a = cut_args(c);
  const int threads = 512;
  int per_sm = 0;
  CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cut_gdp_kernel<4>, threads, 0));
  if (per_sm < 1) return fail(c, F2M_ERR_CUDA, "cut GDP kernel does not fit an SM");
  if (per_sm > 2) per_sm = 2;
  const int grid = c->num_sms * per_sm;
  CK(c, cudaMemsetAsync(c->d_gdp, 0, sizeof(GdpCtl), c->st));
  cudaEvent_t e0 = c->ev0, e1 = c->ev1;
  CK(c, cudaEventRecord(e0, c->st));
  const int32_t* rp = c->d_rp;
  const int2* ec = c->d_ec;
  const uint8_t* mask = S->d_mask;
  const int32_t* ptr = S->d_ptr;
  const int2* items = S->d_items;
  int32_t M = (int32_t)S->M;
  const int32_t* lcuts = S->d_long;
  int32_t nlong = S->nlong;
  int32_t* l0 = c->d_lam[c->cur];
  int32_t* l1 = c->d_lam[c->cur ^ 1];
  int32_t* m0 = S->d_mu[S->cur];
  int32_t* m1 = S->d_mu[S->cur ^ 1];
  int32_t F = c->p.frac_bits, shift = c->p.damping_shift;
  long long msw = max_sweeps, tcl = tcap, budget = c->p.barrier_budget_cycles;
  GdpCtl* ctl = c->d_gdp;
  void* args[] = {(void*)&rp, (void*)&ec, (void*)&mask, (void*)&a, (void*)&ptr, (void*)&items, (void*)&M,
                  (void*)&lcuts, (void*)&nlong, (void*)&l0, (void*)&l1, (void*)&m0, (void*)&m1, (void*)&F, (void*)&shift, (void*)&msw,
                  (void*)&ctl, (void*)&tb, (void*)&tc, (void*)&tcl, (void*)&budget};
  CK(c, cudaLaunchCooperativeKernel((const void*)cut_gdp_kernel<4>, dim3(grid), dim3(threads), args, 0, c->st));
  count_launch();
  CK(c, cudaEventRecord(e1, c->st));
  GdpCtl h{};
  CK(c, cudaMemcpyAsync(&h, c->d_gdp, sizeof(h), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (ms) {
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms += t;
  }
  *sweeps = h.sweeps;
  // the state after the last sweep that was kept: an overflowing sweep is not
  const bool ovf = (h.status & kGdpOverflow) != 0;
  const long long used = ovf ? h.sweeps - 1 : h.sweeps;
  if (used & 1) {
    c->cur ^= 1;
    S->cur ^= 1;
  }
  c->gdp_kernel = F2M_GDP_KERNEL_CUTS;
  if (h.status & kGdpTimeout) return fail(c, F2M_ERR_TIMEOUT, "device-wide barrier wait exceeded its budget");
  if (ovf) return fail(c, F2M_ERR_OVERFLOW, "|lambda| or a cut dual reached 2^29");
  return h.fixed_point ? F2M_OK : F2M_ERR_NOT_CONVERGED;
}

// bound2 (and rule (7) into d_x2 when want_x) at the current duals with cuts
f2m_status cut_bound_extract(f2m_ctx* c, bool want_x, int64_t* b2, int64_t* bad) {
  CutState* S = c->cuts;
  f2m_status s = cut_lists(c);
  if (s != F2M_OK) return s;
  int32_t fb = 0;
  const int32_t* lam = cur_lambda(c, &fb);
  if (fb != c->p.frac_bits) return fail(c, F2M_ERR_INVALID_ARG, "cut duals are held at F bits");
  CK(c, cudaMemsetAsync(c->d_scalar, 0, sizeof(long long), c->st));
  CK(c, cudaMemsetAsync(c->d_bad, 0, sizeof(unsigned long long), c->st));
  cut_bound_extract_kernel<<<grid_of(c->n, 256), 256, 0, c->st>>>(
      c->d_rp, c->d_ec, S->d_mask, cut_args(c), lam, S->d_mu[S->cur], (int32_t)S->M, fb,
      want_x ? c->d_x2 : nullptr, c->d_scalar, c->d_bad);
  count_launch();
  long long h = 0;
  unsigned long long nb = 0;
  CK(c, cudaMemcpyAsync(&h, c->d_scalar, sizeof(h), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaMemcpyAsync(&nb, c->d_bad, sizeof(nb), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (b2) *b2 = h;
  if (bad) *bad = (int64_t)nb;
  return F2M_OK;
}

// pricing with cuts: the plain scan with lamp (a superset), then the exact test
f2m_status cut_price(f2m_ctx* c, double* ms) {
  CutState* S = c->cuts;
  int32_t fb = 0;
  const int32_t* lam = cur_lambda(c, &fb);
  if (fb != c->p.frac_bits) return fail(c, F2M_ERR_INVALID_ARG, "cut duals are held at F bits");
  const int64_t n1 = c->n + 1;
  if (!S->d_lamp) {
    CK(c, dalloc(&S->d_lamp, c->n));
    CK(c, dalloc(&S->d_small, 4));
  }
  const CutArgs a = cut_args(c);
  CK(c, cudaMemsetAsync(S->d_small, 0, sizeof(int32_t), c->st));
  cut_lamp_kernel<<<grid_of(c->n, 256), 256, 0, c->st>>>(a, lam, S->d_mu[S->cur], S->d_lamp, S->d_small);
  count_launch();
  int32_t ovf = 0;
  CK(c, cudaMemcpyAsync(&ovf, S->d_small, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (ovf) return fail(c, F2M_ERR_OVERFLOW, "lambda plus cut duals exceeds 32 bits");
  f2m_status s = price_internal(c, ms, S->d_lamp);
  if (s != F2M_OK) return s;
  const int64_t np = c->npairs;
  if (np == 0) return F2M_OK;
  if (np > S->pair_cap) {
    dfree(S->d_keep);
    dfree(S->d_kpos);
    dfree(S->d_pairs2);
    dfree(S->d_pscan);
    S->pair_cap = np + np / 4 + 1024;
    if (S->pair_cap >= INT_MAX) return fail(c, F2M_ERR_INVALID_ARG, "too many pricing pairs");
    CK(c, dalloc(&S->d_keep, S->pair_cap + 1));
    CK(c, dalloc(&S->d_kpos, S->pair_cap + 1));
    CK(c, dalloc(&S->d_pairs2, S->pair_cap));
    CK(c, dalloc(&S->d_pscan, (int64_t)scan_scratch_ints((int32_t)S->pair_cap + 1)));
  }
  (void)n1;
  cut_pair_keep_kernel<<<grid_of(np, 256), 256, 0, c->st>>>(c->d_pairs, np, c->d_xy, a, lam, S->d_mu[S->cur], fb,
                                                            S->d_keep);
  count_launch();
  CK(c, launch_scan(S->d_keep, S->d_kpos, (int32_t)np, S->d_pscan, c->st));
  cut_pair_compact_kernel<<<grid_of(np, 256), 256, 0, c->st>>>(c->d_pairs, np, S->d_keep, S->d_kpos, S->d_pairs2);
  count_launch();
  int32_t kept = 0;
  CK(c, cudaMemcpyAsync(&kept, S->d_kpos + np, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (kept > 0)
    CK(c, cudaMemcpyAsync(c->d_pairs, S->d_pairs2, sizeof(int2) * kept, cudaMemcpyDeviceToDevice, c->st));
  c->npairs = kept;
  c->seg_pairs.assign(1, kept);
  return F2M_OK;
}

// components of the support of the x held now as one cut layer: comp [n] on
// the device (d_comp_out), number of cuts in *m_out
f2m_status cut_separate(f2m_ctx* c, int32_t* d_comp_out, int32_t* m_out) {
  if (!c->cuts) c->cuts = new CutState();
  CutState* S = c->cuts;
  const int32_t n = c->n;
  if (!S->d_lab) {
    CK(c, dalloc(&S->d_lab, n));
    CK(c, dalloc(&S->d_cross, n));
    CK(c, dalloc(&S->d_flag, n + 1));
    CK(c, dalloc(&S->d_rank, n + 1));
    if (!S->d_small) CK(c, dalloc(&S->d_small, 4));
    if (S->ptr_cap < n + 1) {
      dfree(S->d_cnt);
      dfree(S->d_ptr);
      dfree(S->d_scan);
      dfree(S->d_lflag);
      dfree(S->d_lpos);
      dfree(S->d_long);
      S->ptr_cap = n + 1;
      CK(c, dalloc(&S->d_cnt, S->ptr_cap));
      CK(c, dalloc(&S->d_ptr, S->ptr_cap));
      CK(c, dalloc(&S->d_scan, (int64_t)scan_scratch_ints((int32_t)S->ptr_cap)));
      CK(c, dalloc(&S->d_lflag, S->ptr_cap));
      CK(c, dalloc(&S->d_lpos, S->ptr_cap));
      CK(c, dalloc(&S->d_long, S->ptr_cap));
      S->built_version = -1;
    }
  }
  const int g = grid_of(n, 256);
  cc_init_kernel<<<g, 256, 0, c->st>>>(S->d_lab, n);
  count_launch();
  // hooking and pointer jumping until no label moves (the labels end at the
  // smallest node of each component); bounded by n rounds
  for (int32_t round = 0;; ++round) {
    if (round > n) return fail(c, F2M_ERR_CUDA, "component labelling did not settle");
    CK(c, cudaMemsetAsync(S->d_small, 0, sizeof(int32_t), c->st));
    cc_hook_kernel<<<g, 256, 0, c->st>>>(c->d_rp, c->d_ec, c->d_x2, n, S->d_lab, S->d_small);
    cc_compress_kernel<<<g, 256, 0, c->st>>>(S->d_lab, n, S->d_small);
    count_launches(2);
    int32_t changed = 0;
    CK(c, cudaMemcpyAsync(&changed, S->d_small, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (!changed) break;
  }
  CK(c, cudaMemsetAsync(S->d_cross, 0, sizeof(int32_t) * n, c->st));
  cc_cross_kernel<<<g, 256, 0, c->st>>>(c->d_rp, c->d_ec, S->d_lab, n, S->d_cross, S->d_flag);
  count_launch();
  CK(c, launch_scan(S->d_flag, S->d_rank, n, S->d_scan, c->st));
  int32_t m = 0;
  CK(c, cudaMemcpyAsync(&m, S->d_rank + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  cc_keep_kernel<<<g, 256, 0, c->st>>>(S->d_lab, S->d_cross, n, m, S->d_flag);
  count_launch();
  CK(c, launch_scan(S->d_flag, S->d_rank, n, S->d_scan, c->st));
  cc_label_kernel<<<g, 256, 0, c->st>>>(S->d_lab, S->d_flag, S->d_rank, n, d_comp_out);
  count_launch();
  int32_t kept = 0;
  CK(c, cudaMemcpyAsync(&kept, S->d_rank + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  *m_out = m >= 2 ? kept : 0;
  if (m < 2) CK(c, cudaMemsetAsync(d_comp_out, 0xff, sizeof(int32_t) * n, c->st));
  return F2M_OK;
}

// appends a layer from device labels; checks them and the crossing counts
f2m_status cut_add_layer(f2m_ctx* c, const int32_t* d_labels, int32_t ncuts) {
  if (!c->cuts) c->cuts = new CutState();
  CutState* S = c->cuts;
  if (S->L >= kMaxCutLayers) return fail(c, F2M_ERR_INVALID_ARG, "at most 8 cut layers");
  if (ncuts < 1) return fail(c, F2M_ERR_INVALID_ARG, "a layer needs at least one cut");
  if (c->seg_off.size() != 2) return fail(c, F2M_ERR_INVALID_ARG, "cuts are for single-instance contexts");
  if (c->d_b) return fail(c, F2M_ERR_INVALID_ARG, "cuts need b_v = 2 (F2M)");
  const int32_t n = c->n;
  if (!S->d_comp) CK(c, dalloc(&S->d_comp, (int64_t)kMaxCutLayers * n));
  if (!S->d_small) CK(c, dalloc(&S->d_small, 4));
  int32_t* dst = S->d_comp + (int64_t)S->L * n;
  CK(c, cudaMemcpyAsync(dst, d_labels, sizeof(int32_t) * n, cudaMemcpyDefault, c->st));
  int32_t big = INT_MAX;
  CK(c, cudaMemcpyAsync(S->d_small, &big, sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
  cut_label_check_kernel<<<grid_of(n, 256), 256, 0, c->st>>>(dst, n, ncuts, S->d_small);
  count_launch();
  int32_t badv = INT_MAX;
  CK(c, cudaMemcpyAsync(&badv, S->d_small, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (badv != INT_MAX)
    return fail(c, F2M_ERR_INVALID_ARG, "cut label outside [-1, ncuts) at node " + std::to_string(badv));
  const int64_t M0 = S->M;
  // the duals: old ones kept, the new layer's at 0 (both halves of the buffer)
  if (M0 + ncuts > S->mu_cap) {
    int32_t* nb[2] = {nullptr, nullptr};
    const int64_t cap = (M0 + ncuts) * 2 + 1024;
    CK(c, dalloc(&nb[0], cap));
    CK(c, dalloc(&nb[1], cap));
    if (M0 > 0) CK(c, cudaMemcpyAsync(nb[0], S->d_mu[S->cur], sizeof(int32_t) * M0, cudaMemcpyDeviceToDevice, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    dfree(S->d_mu[0]);
    dfree(S->d_mu[1]);
    S->d_mu[0] = nb[0];
    S->d_mu[1] = nb[1];
    S->cur = 0;
    S->mu_cap = cap;
  }
  CK(c, cudaMemsetAsync(S->d_mu[S->cur] + M0, 0, sizeof(int32_t) * ncuts, c->st));
  S->L += 1;
  S->ncuts.push_back(ncuts);
  S->off.assign(1, 0);
  for (int32_t v : S->ncuts) S->off.push_back(S->off.back() + v);
  S->M = M0 + ncuts;
  S->built_L = -1;
  f2m_status s = cut_lists(c);
  if (s == F2M_OK) {
    CK(c, cudaMemcpyAsync(S->d_small, &big, sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    cut_short_kernel<<<grid_of(ncuts, 256), 256, 0, c->st>>>(S->d_cnt + M0, ncuts, S->d_small);
    count_launch();
    CK(c, cudaMemcpyAsync(&badv, S->d_small, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (badv != INT_MAX)
      s = fail(c, F2M_ERR_INVALID_ARG,
               "cut " + std::to_string(badv) + " of the new layer has fewer than 3 crossing candidate edges");
  }
  if (s != F2M_OK) {  // take the layer back
    S->L -= 1;
    S->ncuts.pop_back();
    S->off.pop_back();
    S->M = M0;
    S->built_L = -1;
  }
  return s;
}

}  // namespace f2m

using namespace f2m;

extern "C" f2m_status f2m_separate(f2m_ctx* c, int32_t* comp, int32_t* ncuts) {
  if (!c || !ncuts) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  if (c->seg_off.size() != 2) return fail(c, F2M_ERR_INVALID_ARG, "cuts are for single-instance contexts");
  int32_t* d = nullptr;
  CK(c, dalloc(&d, c->n));
  int32_t m = 0;
  f2m_status s = cut_separate(c, d, &m);
  if (s == F2M_OK && comp) {
    cudaError_t e = cudaMemcpyAsync(comp, d, sizeof(int32_t) * c->n, cudaMemcpyDefault, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) s = cuda_fail(c, e, "copy labels");
  }
  cudaStreamSynchronize(c->st);
  dfree(d);
  *ncuts = m;
  return s;
}

extern "C" f2m_status f2m_add_cut_layer(f2m_ctx* c, const int32_t* comp, int32_t ncuts) {
  if (!c || !comp) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  return cut_add_layer(c, comp, ncuts);
}

extern "C" f2m_status f2m_get_cut_duals(f2m_ctx* c, int32_t* mu, int64_t* count, int32_t* layers) {
  if (!c || !count) return fail(c, F2M_ERR_INVALID_ARG, "NULL argument");
  const int64_t cap = *count;
  *count = cut_count(c);
  if (layers) *layers = c->cuts ? c->cuts->L : 0;
  if (!mu || *count == 0) return F2M_OK;
  if (cap < *count) return fail(c, F2M_ERR_INVALID_ARG, "capacity below the number of cuts");
  CK(c, cudaMemcpyAsync(mu, c->cuts->d_mu[c->cuts->cur], sizeof(int32_t) * *count, cudaMemcpyDefault, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return F2M_OK;
}

// The subtour driver: GDP phases with pricing (as f2m_solve's first phase,
// without the finisher), then rounds of separation, a new layer and GDP over
// node and cut duals with pricing, each round ending with rule (7) for the
// next separation.
extern "C" f2m_status f2m_solve_subtour(f2m_ctx* c, int32_t rounds, f2m_subtour_info* info_out) {
  if (!c) return fail(c, F2M_ERR_INVALID_ARG, "NULL context");
  if (rounds < 0 || rounds > kMaxCutLayers) return fail(c, F2M_ERR_INVALID_ARG, "rounds must be in 0..8");
  if (c->seg_off.size() != 2 || c->d_b) return fail(c, F2M_ERR_INVALID_ARG, "single F2M instance only");
  const auto t0 = std::chrono::steady_clock::now();
  f2m_subtour_info info;
  std::memset(&info, 0, sizeof(info));
  info.frac_bits = c->p.frac_bits;
  f2m_status status = F2M_OK;
  int32_t* d_lab = nullptr;
  CK(c, dalloc(&d_lab, c->n));
  // one stage: GDP phases with pricing until a scan finds nothing
  auto stage = [&](int64_t* b2_out) -> f2m_status {
    for (int32_t k = 0;; ++k) {
      int64_t sw = 0;
      f2m_status s = gdp_phase(c, c->p.max_iters, &sw, false, 0, &info.ms_gdp);
      info.iterations += sw;
      info.phases += 1;
      if (s != F2M_OK && s != F2M_ERR_NOT_CONVERGED) return s;
      if (!c->p.pricing) break;
      if (info.pricing_rounds >= c->p.max_pricing_rounds) return fail(c, F2M_ERR_NOT_CONVERGED, "pricing rounds exhausted");
      s = cut_count(c) ? cut_price(c, &info.ms_pricing) : price_internal(c, &info.ms_pricing, nullptr);
      if (s != F2M_OK) return s;
      info.pricing_rounds += 1;
      if (c->npairs == 0) break;
      const int64_t found = c->npairs;
      s = merge_internal(c, c->d_pairs, c->npairs, &info.ms_merge);
      if (s != F2M_OK) return s;
      info.edges_added += found;
    }
    int64_t bad = 0;
    f2m_status s = cut_count(c) ? cut_bound_extract(c, true, b2_out, &bad) : extract_internal(c, &bad, nullptr);
    if (s != F2M_OK) return s;
    if (!cut_count(c)) s = bound_internal(c, b2_out);
    return s;
  };
  int64_t b2 = 0;
  status = stage(&b2);
  info.bound2_f2m = b2;
  info.bound2 = b2;
  for (int32_t r = 0; r < rounds && status == F2M_OK; ++r) {
    const auto s0 = std::chrono::steady_clock::now();
    int32_t m = 0;
    status = cut_separate(c, d_lab, &m);
    info.ms_separate += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s0).count();
    if (status != F2M_OK || m == 0) break;
    status = cut_add_layer(c, d_lab, m);
    if (status != F2M_OK) break;
    info.rounds += 1;
    info.cuts += m;
    status = stage(&b2);
    info.bound2 = b2;
  }
  dfree(d_lab);
  info.layers = c->cuts ? c->cuts->L : 0;
  info.certified = status == F2M_OK && c->p.pricing ? 1 : 0;
  info.status = status;
  info.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info_out) *info_out = info;
  return status;
}
