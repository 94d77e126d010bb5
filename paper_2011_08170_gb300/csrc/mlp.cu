// Warm-start network 16 -> 128 -> 128 -> 1 (ReLU) on the tensor cores.
//
// The paper's iteration (Section 3) may start from any lambda; this network
// predicts lambda_v / s_v from node v's sorted 16 nearest-neighbour distances
// (divided by s_v = max(1, their mean)), and the solver starts from
// lambda0_v = rint(2^F s_v y_v).  GDP then runs exactly as from a cold start.
//
// Every matrix product is one tcgen05.mma chain (kind::f16, bf16 operands in
// shared memory, fp32 accumulators in tensor memory) over a tile of 128
// samples; one thread issues the MMAs, and the 128 threads of the CTA run the
// epilogues, thread b owning sample b (tensor-memory lane b).  Products per
// tile (D = A B^T, A: M x K, B: N x K, both K-major):
//   forward   D1 = F W1^T            (128 x 128, K 16)    -> z1, h1 = bf16(relu)
//             D2 = H1 W2^T           (128 x 128, K 128)   -> z2, y = relu(z2) w3 + b3
//   backward  [dW2 | db2] += dZ2^T [H1 | 1]  (128 x 144, K = samples)
//             dH1 = dZ2 W2           (128 x 128, K 128)   (B operand: W2 transposed)
//             dW3 += H2^T dY         (128 x 16, K = samples; column 0 used)
//             [dW1 | db1] += dZ1^T [F | 1]   (128 x 32, K = samples)
// The weight-gradient accumulators stay in tensor memory across the CTA's
// tiles; each CTA writes one partial gradient, and mlp_reduce_kernel sums the
// partials in a fixed order and applies Adam (fp32 master weights), then
// refreshes the bf16 operand images of W1, W2 and W2^T.
#include <climits>
#include <cmath>

#include "f2m_device.cuh"
#include "f2m_internal.h"
#include "tcgen05.cuh"

namespace f2m {

namespace {

using tc::kmajor_off;

constexpr int kTile = 128;
constexpr long long kWaitLimit = 1LL << 24;  // mbarrier polls before giving up

// shared-memory layout of the training kernel (bytes)
constexpr int kSW1 = 0;                       // B of D1: W1 [128 x 16]
constexpr int kSW2 = kSW1 + kImgW1Bytes;      // B of D2: W2 [128 x 128]
constexpr int kSW2T = kSW2 + kImgW2Bytes;     // B of dH1: W2^T [128 x 128]
constexpr int kSF = kSW2T + kImgW2Bytes;      // A of D1: F [128 x 16]
constexpr int kSFT = kSF + 128 * 16 * 2;      // B of dW1: [F | 1]^T [32 x 128]
constexpr int kSR1 = kSFT + 32 * 128 * 2;     // A of D2 (H1) then of dH1 (dZ2) [128 x 128]
constexpr int kSH1T = kSR1 + 128 * 128 * 2;   // B of dW2: [H1 | 1]^T [144 x 128]
constexpr int kSR2 = kSH1T + 144 * 128 * 2;   // A of dW2 (dZ2^T) then of dW1 (dZ1^T) [128 x 128]
constexpr int kSH2T = kSR2 + 128 * 128 * 2;   // A of dW3: H2^T [128 x 128]
constexpr int kSDY = kSH2T + 128 * 128 * 2;   // B of dW3: [dY | 0]^T [16 x 128]
constexpr int kSBias = kSDY + 16 * 128 * 2;   // b1, b2, w3 (fp32, 3 x 128)
constexpr int kSRed = kSBias + 3 * 128 * 4;   // 4 warps x 2 floats
constexpr int kSMbar = kSRed + 64;            // one mbarrier
constexpr int kSTmem = kSMbar + 8;            // tensor-memory address
constexpr int kTrainSmem = kSTmem + 8;

// tensor-memory columns of the training kernel (512 allocated)
constexpr uint32_t kC_D1 = 0, kC_D2 = 128, kC_dW2 = 256, kC_dW1 = 416, kC_dW3 = 448;

// forward-only kernel: W1, W2, F, H1, biases
constexpr int kFW1 = 0;
constexpr int kFW2 = kFW1 + kImgW1Bytes;
constexpr int kFF = kFW2 + kImgW2Bytes;
constexpr int kFH = kFF + 128 * 16 * 2;
constexpr int kFBias = kFH + 128 * 128 * 2;
constexpr int kFMbar = kFBias + 3 * 128 * 4;
constexpr int kFTmem = kFMbar + 8;
// 80 KB so that at most two CTAs (2 x 256 tensor-memory columns) share an SM
constexpr int kFwdSmem = 80 * 1024;
static_assert(kFTmem + 8 <= kFwdSmem, "forward shared memory");
static_assert(kTrainSmem <= 227 * 1024, "training shared memory");

__device__ __forceinline__ void copy16(uint8_t* dst, const uint8_t* src, int bytes, int tid, int nthreads) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = tid; i < bytes / 16; i += nthreads) d[i] = s[i];
}

// row b of a K-major tile with 128 columns, 32 columns starting at c0
__device__ __forceinline__ void store_row32(uint8_t* tile, int b, int c0, const float (&v)[32]) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    uint4 q;
    q.x = tc::pack_bf16x2(v[8 * g + 0], v[8 * g + 1]);
    q.y = tc::pack_bf16x2(v[8 * g + 2], v[8 * g + 3]);
    q.z = tc::pack_bf16x2(v[8 * g + 4], v[8 * g + 5]);
    q.w = tc::pack_bf16x2(v[8 * g + 6], v[8 * g + 7]);
    *reinterpret_cast<uint4*>(tile + kmajor_off(b, c0 + 8 * g, 128)) = q;
  }
}

// column b of a K-major tile with 128 columns (the transposed copy): rows c0..c0+31
__device__ __forceinline__ void store_col32(uint8_t* tile, int b, int c0, const float (&v)[32]) {
#pragma unroll
  for (int i = 0; i < 32; ++i)
    *reinterpret_cast<unsigned short*>(tile + kmajor_off(c0 + i, b, 128)) = tc::bf16_bits(v[i]);
}

// features of sample row b into F [128 x 16] (row b) and, if ft, into [F|1]^T (column b)
__device__ __forceinline__ void load_features(const float* __restrict__ feat, long long s, bool valid,
                                              uint8_t* sF, uint8_t* sFT, int b) {
  float f[16];
  if (valid) {
    const float4* p = reinterpret_cast<const float4*>(feat + s * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = __ldg(p + q);
      f[4 * q] = t.x; f[4 * q + 1] = t.y; f[4 * q + 2] = t.z; f[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) f[j] = 0.f;
  }
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    uint4 q;
    q.x = tc::pack_bf16x2(f[8 * g + 0], f[8 * g + 1]);
    q.y = tc::pack_bf16x2(f[8 * g + 2], f[8 * g + 3]);
    q.z = tc::pack_bf16x2(f[8 * g + 4], f[8 * g + 5]);
    q.w = tc::pack_bf16x2(f[8 * g + 6], f[8 * g + 7]);
    *reinterpret_cast<uint4*>(sF + kmajor_off(b, 8 * g, 16)) = q;
  }
  if (sFT) {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      *reinterpret_cast<unsigned short*>(sFT + kmajor_off(j, b, 128)) = tc::bf16_bits(f[j]);
  }
}

__device__ __forceinline__ uint32_t tmem_at(uint32_t base, int warp, uint32_t col) {
  return base + ((uint32_t)(warp * 32) << 16) + col;
}

// one thread: the chain of k-steps of one product
__device__ __forceinline__ void mma_chain(uint32_t d, uint32_t a, int akdim, uint32_t b, int bkdim,
                                          int ksteps, uint32_t idesc, bool acc_first) {
  for (int s = 0; s < ksteps; ++s)
    tc::mma_bf16(d, tc::smem_desc(a + 256 * s, akdim), tc::smem_desc(b + 256 * s, bkdim), idesc,
                 (s > 0 || acc_first) ? 1u : 0u);
}

// Wait for the commit of the current phase; on a timeout every thread learns it
// after the barrier and the kernel stops.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t& phase, int* s_abort, int* status) {
  const bool ok = tc::mbar_wait(mbar, phase, kWaitLimit);
  phase ^= 1u;
  if (!ok) {
    *s_abort = 1;
    atomicOr(status, 1);
  }
  __syncthreads();
  tc::fence_after();
  return *s_abort == 0;
}

// --------------------------------------------------------------------------------------
// forward (inference); optionally lambda0 = rint(2^F s y), clamped to |lambda0| <= 2^27
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1)
mlp_forward_kernel(const uint8_t* __restrict__ img, const float* __restrict__ master,
                   const float* __restrict__ feat, long long count, float* __restrict__ y_out,
                   const float* __restrict__ scale, int32_t* __restrict__ lam_out, int32_t F,
                   int* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5;
  uint8_t* sW1 = smem + kFW1;
  uint8_t* sW2 = smem + kFW2;
  uint8_t* sF = smem + kFF;
  uint8_t* sH = smem + kFH;
  float* sb1 = reinterpret_cast<float*>(smem + kFBias);
  float* sb2 = sb1 + 128;
  float* sw3 = sb2 + 128;
  const uint32_t mbar = tc::smem_u32(smem + kFMbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kFTmem);

  if (tid == 0) {
    s_abort = 0;
    tc::mbar_init(mbar, 1);
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 256);
  copy16(sW1, img, kImgW1Bytes, tid, 128);
  copy16(sW2, img + kImgW1Bytes, kImgW2Bytes, tid, 128);
  sb1[tid] = master[kOb1 + tid];
  sb2[tid] = master[kOb2 + tid];
  sw3[tid] = master[kOw3 + tid];
  const float b3 = master[kOb3];
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  const uint32_t aF = tc::smem_u32(sF), aW1 = tc::smem_u32(sW1), aH = tc::smem_u32(sH),
                 aW2 = tc::smem_u32(sW2);

  for (long long t0 = (long long)blockIdx.x * kTile; t0 < count; t0 += (long long)gridDim.x * kTile) {
    const long long s = t0 + tid;
    const bool valid = s < count;
    load_features(feat, s, valid, sF, nullptr, tid);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_chain(tmem + kC_D1, aF, 16, aW1, 16, 1, tc::idesc_bf16(128, 128), false);
      tc::commit(mbar);
    }
    if (!wait_phase(mbar, phase, &s_abort, status)) break;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      float v[32];
      tc::tmem_ld32(tmem_at(tmem, warp, kC_D1 + 32 * q), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i] + sb1[32 * q + i], 0.f);
      store_row32(sH, tid, 32 * q, v);
    }
    tc::fence_before();
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_chain(tmem + kC_D2, aH, 128, aW2, 128, 8, tc::idesc_bf16(128, 128), false);
      tc::commit(mbar);
    }
    if (!wait_phase(mbar, phase, &s_abort, status)) break;
    float y = b3;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      float v[32];
      tc::tmem_ld32(tmem_at(tmem, warp, kC_D2 + 32 * q), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) y = fmaf(fmaxf(v[i] + sb2[32 * q + i], 0.f), sw3[32 * q + i], y);
    }
    if (valid) {
      if (y_out) y_out[s] = y;
      if (lam_out) {
        float l = ldexpf(scale[s] * y, F);
        l = (l == l) ? fminf(fmaxf(l, -(float)kLambda0Limit), (float)kLambda0Limit) : 0.f;
        lam_out[s] = __float2int_rn(l);
      }
    }
    tc::fence_before();
    __syncthreads();
  }
  // nothing of this CTA is in flight here: every commit was waited for, or the
  // wait gave up and the CTA stops either way
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// --------------------------------------------------------------------------------------
// forward + backward over the CTA's tiles of one step; partial gradient per CTA
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1)
mlp_train_kernel(const uint8_t* __restrict__ img, const float* __restrict__ master,
                 const float* __restrict__ feat, const float* __restrict__ target,
                 const int32_t* __restrict__ perm, long long s0, long long count, float two_over_b,
                 float* __restrict__ partial, long long* step_ctr, int* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* sW1 = smem + kSW1;
  uint8_t* sW2 = smem + kSW2;
  uint8_t* sW2T = smem + kSW2T;
  uint8_t* sF = smem + kSF;
  uint8_t* sFT = smem + kSFT;
  uint8_t* sR1 = smem + kSR1;
  uint8_t* sH1T = smem + kSH1T;
  uint8_t* sR2 = smem + kSR2;
  uint8_t* sH2T = smem + kSH2T;
  uint8_t* sDY = smem + kSDY;
  float* sb1 = reinterpret_cast<float*>(smem + kSBias);
  float* sb2 = sb1 + 128;
  float* sw3 = sb2 + 128;
  float* sred = reinterpret_cast<float*>(smem + kSRed);
  const uint32_t mbar = tc::smem_u32(smem + kSMbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kSTmem);

  if (tid == 0) {
    s_abort = 0;
    tc::mbar_init(mbar, 1);
    if (blockIdx.x == 0 && step_ctr) *step_ctr += 1;  // Adam step number read by the reduce kernel
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  copy16(sW1, img, kImgW1Bytes, tid, 128);
  copy16(sW2, img + kImgW1Bytes, kImgW2Bytes, tid, 128);
  copy16(sW2T, img + kImgW1Bytes + kImgW2Bytes, kImgW2Bytes, tid, 128);
  sb1[tid] = master[kOb1 + tid];
  sb2[tid] = master[kOb2 + tid];
  sw3[tid] = master[kOw3 + tid];
  const float b3 = master[kOb3];
  // constant rows: the ones row of [H1 | 1]^T (row 128) and [F | 1]^T (row 16),
  // zero rows 129..143, 17..31 and 1..15 of [dY | 0]^T
  const unsigned short one = tc::bf16_bits(1.f);
  for (int r = 128; r < 144; ++r)
    *reinterpret_cast<unsigned short*>(sH1T + kmajor_off(r, tid, 128)) = r == 128 ? one : 0;
  for (int r = 16; r < 32; ++r)
    *reinterpret_cast<unsigned short*>(sFT + kmajor_off(r, tid, 128)) = r == 16 ? one : 0;
  for (int r = 1; r < 16; ++r) *reinterpret_cast<unsigned short*>(sDY + kmajor_off(r, tid, 128)) = 0;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  const uint32_t aW1 = tc::smem_u32(sW1), aW2 = tc::smem_u32(sW2), aW2T = tc::smem_u32(sW2T),
                 aF = tc::smem_u32(sF), aFT = tc::smem_u32(sFT), aR1 = tc::smem_u32(sR1),
                 aH1T = tc::smem_u32(sH1T), aR2 = tc::smem_u32(sR2), aH2T = tc::smem_u32(sH2T),
                 aDY = tc::smem_u32(sDY);
  constexpr uint32_t id128 = tc::idesc_bf16(128, 128), id144 = tc::idesc_bf16(128, 144),
                     id32 = tc::idesc_bf16(128, 32), id16 = tc::idesc_bf16(128, 16);
  float loss = 0.f, db3 = 0.f;
  bool any = false;

  for (long long t0 = (long long)blockIdx.x * kTile; t0 < count; t0 += (long long)gridDim.x * kTile) {
    const long long pos = t0 + tid;
    const bool valid = pos < count;
    const long long s = valid ? (perm ? (long long)perm[s0 + pos] : s0 + pos) : 0;
    load_features(feat, s, valid, sF, sFT, tid);
    const float tgt = valid ? target[s] : 0.f;
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_chain(tmem + kC_D1, aF, 16, aW1, 16, 1, id128, false);
      tc::commit(mbar);
    }
    if (!wait_phase(mbar, phase, &s_abort, status)) break;
    // epilogue 1: z1 -> mask, h1 = bf16(relu(z1)) into H1 (row) and [H1 | 1]^T (column)
    uint32_t mask1[4];
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      float v[32];
      tc::tmem_ld32(tmem_at(tmem, warp, kC_D1 + 32 * q), v);
      uint32_t m = 0;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float z = v[i] + sb1[32 * q + i];
        m |= (z > 0.f ? 1u : 0u) << i;
        v[i] = fmaxf(z, 0.f);
      }
      mask1[q] = m;
      store_row32(sR1, tid, 32 * q, v);
      store_col32(sH1T, tid, 32 * q, v);
    }
    tc::fence_before();
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_chain(tmem + kC_D2, aR1, 128, aW2, 128, 8, id128, false);
      tc::commit(mbar);
    }
    if (!wait_phase(mbar, phase, &s_abort, status)) break;
    // epilogue 2: y, dy; h2 into H2^T; dz2 = bf16(dy w3 [z2 > 0]) into dZ2 (row) and dZ2^T (column)
    float y = b3;
    uint32_t mask2[4];
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      float v[32];
      tc::tmem_ld32(tmem_at(tmem, warp, kC_D2 + 32 * q), v);
      uint32_t m = 0;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float z = v[i] + sb2[32 * q + i];
        m |= (z > 0.f ? 1u : 0u) << i;
        v[i] = fmaxf(z, 0.f);
        y = fmaf(v[i], sw3[32 * q + i], y);
      }
      mask2[q] = m;
      store_col32(sH2T, tid, 32 * q, v);
    }
    const float r = valid ? y - tgt : 0.f;
    const float dy = two_over_b * r;
    loss = fmaf(r, r, loss);
    db3 += dy;
    *reinterpret_cast<unsigned short*>(sDY + kmajor_off(0, tid, 128)) = tc::bf16_bits(dy);
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = ((mask2[q] >> i) & 1u) ? dy * sw3[32 * q + i] : 0.f;
      store_row32(sR1, tid, 32 * q, v);  // D2 is complete: H1 is no longer needed as an operand
      store_col32(sR2, tid, 32 * q, v);
    }
    tc::fence_before();
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_chain(tmem + kC_dW2, aR2, 128, aH1T, 128, 8, id144, any);
      mma_chain(tmem + kC_D1, aR1, 128, aW2T, 128, 8, id128, false);
      mma_chain(tmem + kC_dW3, aH2T, 128, aDY, 128, 8, id16, any);
      tc::commit(mbar);
    }
    if (!wait_phase(mbar, phase, &s_abort, status)) break;
    // epilogue 3: dz1 = bf16(dh1 [z1 > 0]) into dZ1^T (column)
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      float v[32];
      tc::tmem_ld32(tmem_at(tmem, warp, kC_D1 + 32 * q), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = ((mask1[q] >> i) & 1u) ? v[i] : 0.f;
      store_col32(sR2, tid, 32 * q, v);
    }
    tc::fence_before();
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_chain(tmem + kC_dW1, aR2, 128, aFT, 128, 8, id32, any);
      tc::commit(mbar);
    }
    if (!wait_phase(mbar, phase, &s_abort, status)) break;
    any = true;
  }

  // partial gradient of this CTA: row `tid` of each accumulator
  float* out = partial + (size_t)blockIdx.x * (kMlpParams + 1);
  if (s_abort == 0) {
    if (any) {
      for (int q = 0; q < 5; ++q) {  // [dW2 | db2]: columns 0..143 used
        float v[32];
        tc::tmem_ld32(tmem_at(tmem, warp, kC_dW2 + 32 * q), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int c = 32 * q + i;
          if (c < 128) out[kOW2 + tid * 128 + c] = v[i];
          else if (c == 128) out[kOb2 + tid] = v[i];
        }
      }
      float v[32];
      tc::tmem_ld32(tmem_at(tmem, warp, kC_dW1), v);
#pragma unroll
      for (int j = 0; j < 16; ++j) out[kOW1 + tid * 16 + j] = v[j];
      out[kOb1 + tid] = v[16];
      tc::tmem_ld32(tmem_at(tmem, warp, kC_dW3), v);
      out[kOw3 + tid] = v[0];
    } else {
      for (int c = 0; c < 128; ++c) out[kOW2 + tid * 128 + c] = 0.f;
      for (int j = 0; j < 16; ++j) out[kOW1 + tid * 16 + j] = 0.f;
      out[kOb1 + tid] = 0.f;
      out[kOb2 + tid] = 0.f;
      out[kOw3 + tid] = 0.f;
    }
    loss = warp_sum_f(loss);
    db3 = warp_sum_f(db3);
    if (lane == 0) {
      sred[2 * warp] = loss;
      sred[2 * warp + 1] = db3;
    }
    __syncthreads();
    if (tid == 0) {
      out[kOb3] = sred[1] + sred[3] + sred[5] + sred[7];
      out[kMlpParams] = sred[0] + sred[2] + sred[4] + sred[6];
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Sum the per-CTA partials in CTA order; then either store the gradient (and
// loss) or apply one Adam step and refresh the bf16 operand images.
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int nparts, float* __restrict__ grad,
                                  float* master, float* m1, float* m2, uint8_t* __restrict__ img,
                                  const long long* step_ctr, MlpAdam hp, float* loss_log) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kMlpParams) return;
  float g = 0.f;
  for (int c = 0; c < nparts; ++c) g += partial[(size_t)c * (kMlpParams + 1) + p];
  if (p == kMlpParams) {  // loss sum of the step
    if (loss_log) loss_log[step_ctr ? *step_ctr - 1 - hp.log_base : 0] = g;
    return;
  }
  if (grad) {
    grad[p] = g;
    return;
  }
  const long long t = *step_ctr;
  const float frac = hp.total_steps > 1 ? (float)(t - 1) / (float)(hp.total_steps - 1) : 0.f;
  const float lr = hp.lr * (1.f - (1.f - hp.lr_final_frac) * frac);
  const float a = hp.beta1 * m1[p] + (1.f - hp.beta1) * g;
  const float b = hp.beta2 * m2[p] + (1.f - hp.beta2) * g * g;
  m1[p] = a;
  m2[p] = b;
  const float mh = a / (1.f - powf(hp.beta1, (float)t));
  const float vh = b / (1.f - powf(hp.beta2, (float)t));
  const float w = master[p] - lr * mh / (sqrtf(vh) + hp.eps);
  master[p] = w;
  const unsigned short h = tc::bf16_bits(w);
  if (p < kOW1 + 2048) {
    const int i = p / 16, j = p % 16;
    *reinterpret_cast<unsigned short*>(img + kmajor_off(i, j, 16)) = h;
  } else if (p >= kOW2 && p < kOW2 + 16384) {
    const int c = (p - kOW2) / 128, i = (p - kOW2) % 128;
    *reinterpret_cast<unsigned short*>(img + kImgW1Bytes + kmajor_off(c, i, 128)) = h;
    *reinterpret_cast<unsigned short*>(img + kImgW1Bytes + kImgW2Bytes + kmajor_off(i, c, 128)) = h;
  }
}

// bf16 operand images of W1, W2 and W2^T from the fp32 master weights
__global__ void mlp_pack_kernel(const float* __restrict__ master, uint8_t* __restrict__ img) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < 2048) {
    *reinterpret_cast<unsigned short*>(img + kmajor_off(p / 16, p % 16, 16)) = tc::bf16_bits(master[kOW1 + p]);
  } else if (p < 2048 + 16384) {
    const int q = p - 2048, c = q / 128, i = q % 128;
    const unsigned short h = tc::bf16_bits(master[kOW2 + q]);
    *reinterpret_cast<unsigned short*>(img + kImgW1Bytes + kmajor_off(c, i, 128)) = h;
    *reinterpret_cast<unsigned short*>(img + kImgW1Bytes + kImgW2Bytes + kmajor_off(i, c, 128)) = h;
  }
}

// shuffle keys: SplitMix64 of (seed, epoch, position)
__global__ void mlp_perm_keys_kernel(uint64_t key, long long n, uint64_t* __restrict__ keys,
                                     int32_t* __restrict__ idx) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  keys[i] = z ^ (z >> 31);
  idx[i] = (int32_t)i;
}

}  // namespace

cudaError_t mlp_pack(const float* master, uint8_t* img, cudaStream_t st) {
  mlp_pack_kernel<<<(2048 + 16384 + 255) / 256, 256, 0, st>>>(master, img);
  count_launch();
  return cudaGetLastError();
}

int mlp_grid(int num_sms, long long count) {
  long long tiles = (count + kTile - 1) / kTile;
  if (tiles < 1) tiles = 1;
  return (int)(tiles < num_sms ? tiles : num_sms);
}

cudaError_t mlp_forward(const uint8_t* img, const float* master, const float* feat, long long count,
                        float* y, const float* scale, int32_t* lam, int32_t F, int num_sms, int* status,
                        cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
  if (e != cudaSuccess) return e;
  if (count <= 0) return cudaSuccess;
  long long tiles = (count + kTile - 1) / kTile;
  const int grid = (int)(tiles < 2LL * num_sms ? tiles : 2LL * num_sms);
  mlp_forward_kernel<<<grid, 128, kFwdSmem, st>>>(img, master, feat, count, y, scale, lam, F, status);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_train_launch(const uint8_t* img, const float* master, const float* feat, const float* target,
                             const int32_t* perm, long long s0, long long count, float two_over_b,
                             float* partial, int grid, long long* step_ctr, int* status, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem);
  if (e != cudaSuccess) return e;
  mlp_train_kernel<<<grid, 128, kTrainSmem, st>>>(img, master, feat, target, perm, s0, count, two_over_b,
                                                  partial, step_ctr, status);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_reduce_launch(const float* partial, int nparts, float* grad, float* master, float* m1,
                              float* m2, uint8_t* img, const long long* step_ctr, const MlpAdam& hp,
                              float* loss_log, cudaStream_t st) {
  mlp_reduce_kernel<<<(kMlpParams + 1 + 255) / 256, 256, 0, st>>>(partial, nparts, grad, master, m1, m2, img,
                                                                   step_ctr, hp, loss_log);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_perm_keys(uint64_t key, long long n, uint64_t* keys, int32_t* idx, cudaStream_t st) {
  mlp_perm_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(key, n, keys, idx);
  count_launch();
  return cudaGetLastError();
}

}  // namespace f2m
