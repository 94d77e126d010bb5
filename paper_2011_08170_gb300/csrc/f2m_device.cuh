// Device helpers shared by the f2m kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace f2m {

// Edge cost c(u,v): the nearest integer to sqrt(d2), d2 = dx^2 + dy^2 (TSPLIB
// EUC_2D, the input convention of Section 5.1).  Integer-exact: s is the floor
// of sqrt(4*d2) (a double square root as first guess, then corrected in
// integers), and nint(sqrt(d2)) = floor((s + 1) / 2).  No tie exists: an
// integer d2 never equals (r + 1/2)^2.
__device__ __forceinline__ int32_t exact_cost(int32_t dx, int32_t dy) {
  long long d2 = (long long)dx * dx + (long long)dy * dy;
  long long q = 4 * d2;  // < 2^43, exact in double
  long long s = (long long)sqrt((double)q);
  while (s * s > q) --s;
  while ((s + 1) * (s + 1) <= q) ++s;
  return (int32_t)((s + 1) >> 1);
}

__device__ __forceinline__ int32_t exact_cost(int2 a, int2 b) { return exact_cost(a.x - b.x, a.y - b.y); }

// Keep the three smallest values seen, a <= b <= c (values only; ties are
// irrelevant to Eq. 10, which needs the 2nd and 3rd values, not the edges).
__device__ __forceinline__ void top3_insert(int z, int& a, int& b, int& c) {
  if (z < c) {
    c = z;
    if (c < b) { int t = b; b = c; c = t; }
    if (b < a) { int t = a; a = b; b = t; }
  }
}

// Branch-free form of the same insertion: the three smallest of {a, b, c, z}.
__device__ __forceinline__ void top3_insert_minmax(int z, int& a, int& b, int& c) {
  c = min(c, max(b, z));
  b = min(b, max(a, z));
  a = min(a, z);
}

// Eq. 10 step: trunc((z2 + z3) / 2^shift) toward zero, exactly, by shifts
// (a 64-bit division by a run-time divisor is a long software routine)
__device__ __forceinline__ long long gdp_step(int z2, int z3, int shift) {
  const long long s = (long long)z2 + (long long)z3;
  return s >= 0 ? (s >> shift) : -((-s) >> shift);
}

// Top-3 of two partial top-3 sets (each ascending): the 3 smallest of their union.
__device__ __forceinline__ void top3_merge(int a1, int b1, int c1, int& a, int& b, int& c) {
  top3_insert_minmax(a1, a, b, c);
  top3_insert_minmax(b1, a, b, c);
  top3_insert_minmax(c1, a, b, c);
}

// Load that bypasses L1: lambda is rewritten by other SMs between sweeps.
__device__ __forceinline__ int ld_cg(const int* p) { return __ldcg(p); }

// Device-wide barrier for a cooperative launch, bounded: a block whose wait
// runs past `budget` clock cycles gives up and reports false.  One arrival
// counter plus a generation word; the last block to arrive resets the counter
// and bumps the generation.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* gen,
                                             unsigned int nblocks, long long budget) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = gen;
    unsigned int g = *vgen;
    __threadfence();
    unsigned int prev = atomicAdd(count, 1u);
    if (prev == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > budget) { ok = 0; break; }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Device-wide barrier on a monotone arrival counter (cooperative launch only).
// Barrier number k (k = 1, 2, ...) completes when the counter reaches
// k * gridDim.x.  Arrival is one release-ordered atomic add (it publishes the
// block's earlier writes); waiting is acquire-ordered polling of the counter,
// bounded by `budget` clock cycles (false on time-out).  The counter never
// needs resetting, so the last block to arrive does no extra work.
__device__ __forceinline__ bool grid_barrier_counted(unsigned int* count, unsigned int target,
                                                     long long budget) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int v;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(v) : "l"(count) : "memory");
    v += 1;
    if ((int)(v - target) < 0) {
      const long long t0 = clock64();
      for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
        if ((int)(v - target) >= 0) break;
        if (clock64() - t0 > budget) { ok = 0; break; }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Split form of the counted barrier, for thread 0 of each block: arrive
// publishes this block's earlier writes (release) without waiting for a reply;
// wait polls (acquire) until `target` arrivals, bounded by `budget` cycles.
__device__ __forceinline__ void grid_arrive_counted(unsigned int* count) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
}
__device__ __forceinline__ bool grid_wait_counted(unsigned int* count, unsigned int target,
                                                  long long budget) {
  unsigned int v;
  const long long t0 = clock64();
  for (;;) {
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
    if ((int)(v - target) >= 0) return true;
    if (clock64() - t0 > budget) return false;
  }
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned warp_sum_u(unsigned v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exclusive prefix sum over the block (blockDim.x a multiple of 32, <= 1024);
// s_warp needs 33 ints.  total receives the block sum.
__device__ __forceinline__ int block_exclusive_scan(int x, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? s_warp[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) s_warp[lane] = wi - w;
    if (lane == nw - 1) s_warp[32] = wi;
  }
  __syncthreads();
  total = s_warp[32];
  const int r = s_warp[warp] + inc - x;
  __syncthreads();
  return r;
}

}  // namespace f2m
