// Phase 1 of the exact finisher on the GPU: one warp per block of nodes.
//
// The same searches as the host's first blocked phase (finisher.cpp), in the
// same order, so the flow, the potentials and the surpluses it leaves are
// those of the host's phase 1 bit for bit: a block's sources in key order
// (L_i before R_i, i ascending), Dijkstra on reduced costs with the heap
// ordered by (distance, key), searches kept inside the block -- a heap item of
// an outside node coming to the top, or an empty heap, drops the search with
// nothing changed -- and arcs into outside nodes priced at the potentials of
// the phase's start (lambda for a left copy, -lambda for a right one).  The
// arcs and potentials a block reads are written by that block alone, so the
// blocks run independently.
//
// In a warp, lane 0 owns the heap (in shared memory, moved to the block's
// region of global memory when a search outgrows it) and pops;
// the lanes relax the settled node's row in parallel (a row's columns are
// distinct, so their updates do not collide) and hand their pushes to lane 0
// in lane order; the pop order does not depend on the push order, the heap
// order being total up to identical items.  Every search pushes at most
// twice the block's entries plus one items, the size of its heap.  A block
// that runs past its clock budget stops and raises the error flag.
#include <climits>

#include "f2m_device.cuh"
#include "f2m_internal.h"

namespace f2m {

namespace {

struct FinItem {
  long long d;
  int key;
  int node;
};

__device__ __forceinline__ bool fin_less(const FinItem& a, const FinItem& b) {
  return a.d < b.d || (a.d == b.d && a.key < b.key);
}

__device__ __forceinline__ void heap_push(FinItem* h, int& hs, const FinItem& it) {
  int i = hs++;
  h[i] = it;
  while (i > 0) {
    const int p = (i - 1) >> 1;
    if (!fin_less(h[i], h[p])) break;
    const FinItem t = h[i];
    h[i] = h[p];
    h[p] = t;
    i = p;
  }
}

__device__ __forceinline__ FinItem heap_pop(FinItem* h, int& hs) {
  const FinItem top = h[0];
  h[0] = h[--hs];
  int i = 0;
  for (;;) {
    const int l = 2 * i + 1, r = l + 1;
    int s = i;
    if (l < hs && fin_less(h[l], h[s])) s = l;
    if (r < hs && fin_less(h[r], h[s])) s = r;
    if (s == i) break;
    const FinItem t = h[i];
    h[i] = h[s];
    h[s] = t;
    i = s;
  }
  return top;
}

__device__ __forceinline__ FinItem shfl_item(const FinItem& x, int src) {
  FinItem r;
  r.d = __shfl_sync(0xffffffffu, x.d, src);
  r.key = __shfl_sync(0xffffffffu, x.key, src);
  r.node = __shfl_sync(0xffffffffu, x.node, src);
  return r;
}

constexpr int kWarps = 2;         // warps (blocks of nodes) per CTA
constexpr int kSmemHeap = 1024;   // heap items a warp keeps in shared memory

__global__ void __launch_bounds__(32 * kWarps)
fin_block_kernel(int32_t n, const int2* __restrict__ blocks, int32_t nblocks, const int32_t* __restrict__ irp,
                 const int2* __restrict__ iec, const int32_t* __restrict__ twin, uint8_t* y,
                 const int32_t* __restrict__ exl, const int32_t* __restrict__ lam, int32_t F, long long* pi,
                 long long* dist, int32_t* excess, int32_t* via, int32_t* pred, uint32_t* reached,
                 uint32_t* closed, FinItem* heaps, const long long* __restrict__ heap_off, int32_t* orders,
                 long long* pushes_out, int32_t* status, long long budget) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int blk = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (blk >= nblocks) return;
  const int lo = blocks[blk].x, hi = blocks[blk].y;
  for (int i = lo + lane; i < hi; i += 32) {
    pi[i] = lam[i];
    pi[n + i] = -(long long)lam[i];
    excess[i] = exl[i];
    excess[n + i] = -exl[i];
    reached[i] = 0;
    reached[n + i] = 0;
    closed[i] = 0;
    closed[n + i] = 0;
  }
  __syncwarp();
  // the heap starts in shared memory; a search whose heap outgrows it moves
  // it to the block's region of global memory (room for every push) and goes
  // on there -- the pops are the same either way
  __shared__ FinItem s_heap[kWarps][kSmemHeap];
  FinItem* const gheap = heaps + heap_off[blk];
  const long long gcap = heap_off[blk + 1] - heap_off[blk];
  FinItem* heap = s_heap[threadIdx.x >> 5];
  long long hcap = kSmemHeap;
  int32_t* order = orders + 2LL * lo;
  auto key_of = [&](int node) { return node < n ? 2 * node : 2 * (node - n) + 1; };
  auto outside = [&](int node) {
    const int i = node < n ? node : node - n;
    return i < lo || i >= hi;
  };
  auto pi0 = [&](int node) { return node < n ? (long long)lam[node] : -(long long)lam[node - n]; };
  const long long t0 = clock64();
  uint32_t round = 0;
  long long pushes = 0;
  int err = 0;
  for (int i = lo; i < hi && !err; ++i) {
    for (int side = 0; side < 2 && !err; ++side) {
      const int s = side == 0 ? i : n + i;  // key order: L_i before R_i
      for (;;) {
        __syncwarp();
        if (excess[s] <= 0) break;
        ++round;
        int hs = 0, ns = 0, t = -1;  // lane 0's
        heap = s_heap[threadIdx.x >> 5];
        hcap = kSmemHeap;
        if (lane == 0) {
          dist[s] = 0;
          reached[s] = round;
          pred[s] = -1;
          heap_push(heap, hs, FinItem{0, key_of(s), s});
        }
        for (;;) {
          int v = -1, stop = 0;
          long long dv = 0, piv = 0;
          if (lane == 0) {
            for (;;) {
              if (hs == 0) { stop = 1; break; }                     // nothing reachable: dropped
              if (clock64() - t0 > budget) { err = 1; stop = 1; break; }
              const FinItem top = heap_pop(heap, hs);
              const int u = top.node;
              if (outside(u)) { stop = 1; break; }                  // dropped
              if (closed[u] == round || top.d != dist[u]) continue;  // stale item
              closed[u] = round;
              if (excess[u] < 0) { t = u; stop = 1; break; }
              order[ns++] = u;
              v = u;
              dv = top.d;
              piv = pi[u];
              break;
            }
          }
          stop = __shfl_sync(full, stop, 0);
          if (stop) break;
          v = __shfl_sync(full, v, 0);
          dv = __shfl_sync(full, dv, 0);
          piv = __shfl_sync(full, piv, 0);
          __syncwarp();  // lane 0's writes of this settle before the lanes read
          const int row = v < n ? v : v - n;
          const int e0 = irp[row], e1 = irp[row + 1];
          for (int base = e0; base < e1; base += 32) {
            const int e = base + lane;
            FinItem cand{0, 0, 0};
            bool has = false;
            if (e < e1) {
              const int2 q = iec[e];
              const long long C = (long long)q.y << F;
              if (v < n) {  // L_v -> R_j along an arc without flow
                if (!y[e]) {
                  const int j = n + q.x;
                  if (outside(j)) {
                    cand = FinItem{dv + C - piv + pi0(j), key_of(j), j};
                    has = true;
                  } else {
                    const long long d = dv + C - piv + pi[j];
                    if (closed[j] != round && (reached[j] != round || d < dist[j])) {
                      reached[j] = round; dist[j] = d; via[j] = e; pred[j] = v;
                      cand = FinItem{d, key_of(j), j};
                      has = true;
                    }
                  }
                }
              } else {  // R_u -> L_x back along the saturated arc x -> u
                const int a = twin[e];
                if (y[a]) {
                  const int j = q.x;
                  if (outside(j)) {
                    cand = FinItem{dv - C - piv + pi0(j), key_of(j), j};
                    has = true;
                  } else {
                    const long long d = dv - C - piv + pi[j];
                    if (closed[j] != round && (reached[j] != round || d < dist[j])) {
                      reached[j] = round; dist[j] = d; via[j] = a; pred[j] = v;
                      cand = FinItem{d, key_of(j), j};
                      has = true;
                    }
                  }
                }
              }
            }
            unsigned m = __ballot_sync(full, has);
            while (m) {
              const int src = __ffs(m) - 1;
              m &= m - 1;
              const FinItem it = shfl_item(cand, src);
              if (lane == 0) {
                if (hs >= hcap && heap != gheap) {  // move to global memory
                  for (int q = 0; q < hs; ++q) gheap[q] = heap[q];
                  heap = gheap;
                  hcap = gcap;
                }
                if (hs >= hcap) err = 1;
                else heap_push(heap, hs, it);
              }
            }
          }
          __syncwarp();
          if (__shfl_sync(full, err, 0)) break;
        }
        err = __shfl_sync(full, err, 0);
        t = __shfl_sync(full, t, 0);
        if (err || t < 0) break;  // a dropped search leaves this source to the next phase
        long long dt = 0;
        if (lane == 0) {
          for (int j = t; j != s; j = pred[j]) y[via[j]] = (uint8_t)(j >= n);  // one unit along the path
          excess[s] -= 1;
          excess[t] += 1;
          ++pushes;
          dt = dist[t];
        }
        dt = __shfl_sync(full, dt, 0);
        ns = __shfl_sync(full, ns, 0);
        __syncwarp();
        for (int k = lane; k < ns; k += 32) {
          const int u = order[k];
          pi[u] += dt - dist[u];
        }
      }
    }
  }
  if (lane == 0) {
    pushes_out[blk] = pushes;
    if (err) atomicOr(status, 1);
  }
}

__global__ void fin_block_caps_kernel(const int2* __restrict__ blocks, int32_t nblocks, const int32_t* __restrict__ irp,
                                      long long* caps) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nblocks;
       k += (long long)gridDim.x * blockDim.x) {
    const int2 b = blocks[k];
    caps[k] = 2LL * (irp[b.y] - irp[b.x]) + 8;
  }
}

}  // namespace

size_t fin_heap_item_bytes() { return sizeof(FinItem); }

cudaError_t launch_fin_block_caps(const int2* blocks, int32_t nblocks, const int32_t* irp, long long* caps,
                                  cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  fin_block_caps_kernel<<<(nblocks + 255) / 256, 256, 0, st>>>(blocks, nblocks, irp, caps);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fin_blocks(int32_t n, const int2* blocks, int32_t nblocks, const int32_t* irp, const int2* iec,
                              const int32_t* twin, uint8_t* y, const int32_t* exl, const int32_t* lam, int32_t F,
                              long long* pi, long long* dist, int32_t* excess, int32_t* via, int32_t* pred,
                              uint32_t* reached, uint32_t* closed, void* heaps, const long long* heap_off,
                              int32_t* orders, long long* pushes, int32_t* status, long long budget,
                              cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  fin_block_kernel<<<(nblocks + kWarps - 1) / kWarps, 32 * kWarps, 0, st>>>(
      n, blocks, nblocks, irp, iec, twin, y, exl, lam, F, pi, dist, excess, via, pred, reached, closed,
      static_cast<FinItem*>(heaps), heap_off, orders, pushes, status, budget);
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
