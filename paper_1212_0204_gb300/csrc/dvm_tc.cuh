// dvm_tc.cuh -- fifth-generation tensor-core (tcgen05) building blocks of the
// regime network: BF16 operands in shared memory, FP32 accumulators in tensor
// memory (TMEM), one thread issuing the MMAs, an mbarrier for completion.
//
// Operand layout in shared memory (K-major, no swizzle): a matrix of R rows
// and K columns (bf16) is stored as 8 x 8 "core matrices" of 128 contiguous
// bytes (8 rows of 16 bytes); element (r, k) sits at
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,   SBO = K * 16,
// i.e. the core matrices along K are adjacent (leading-dimension byte offset
// 128) and the 8-row groups follow each other (stride byte offset K * 16).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace dvm {
namespace tc {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) in the layout above
__device__ __forceinline__ int kmajor_offset(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start, leading byte offset (between core
// matrices along K), stride byte offset (between 8-row groups), descriptor
// version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(const void* start, unsigned lbo, unsigned sbo) {
  const uint64_t a = (uint64_t)((smem_u32(start) >> 4) & 0x3FFFu);
  return a | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16 with BF16 A and B (both K-major) and an
// FP32 accumulator, shape M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(unsigned* dst_smem, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T
__device__ __forceinline__ void mma_bf16(unsigned dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// generic-proxy writes to shared memory become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on phase `parity`: false after 2^31 SM clock cycles (about a
// second); a poll count would not bound the time, the back-off sleeps can
// last far longer than asked
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, unsigned parity) {
  if (mbar_try_wait(mbar, parity)) return true;
  const long long t0 = clock64();
  for (int i = 0;; ++i) {
    if (mbar_try_wait(mbar, parity)) return true;
    if (clock64() - t0 > (1LL << 31)) return false;
    if (i > 64) __nanosleep(32);
  }
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32w .. 32w + 31; taddr carries the lane in its upper half)
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace tc
}  // namespace dvm

namespace dvm {
namespace tc {

// Shared memory of the tensor-core forward pass of the 10-64-64-1 network
// (128 samples per tile).
struct MlpSmem {
  __nv_bfloat16 A1[128 * 16];  // inputs, K padded to 16
  __nv_bfloat16 B1[64 * 16];   // W1 (N = 64 outputs x K = 16)
  __nv_bfloat16 A2[128 * 64];  // first hidden layer
  __nv_bfloat16 B2[64 * 64];   // W2
  float b1[64], b2[64], w3[64], b3;
  uint64_t mbar;
  unsigned tbase;
};

constexpr int kTcThreads = 128;
constexpr unsigned kTmemCols = 128;  // D1: columns 0..63, D2: 64..127

// Per CTA, once: BF16 copies of W1 and W2 in the operand layout, FP32 biases
// and output weights, the mbarrier and 128 TMEM columns (warp 0).
__device__ inline void mlp_tc_setup(MlpSmem& S, const float* __restrict__ P) {
  const int t = threadIdx.x;
  for (int i = t; i < 64 * 16; i += kTcThreads) {
    const int j = i / 16, k = i % 16;
    const float w = k < 10 ? P[j * 10 + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(S.B1) + kmajor_offset(j, k, 16)) =
        __float2bfloat16_rn(w);
  }
  for (int i = t; i < 64 * 64; i += kTcThreads) {
    const int j = i / 64, k = i % 64;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(S.B2) + kmajor_offset(j, k, 64)) =
        __float2bfloat16_rn(P[704 + i]);
  }
  if (t < 64) {
    S.b1[t] = P[640 + t];
    S.b2[t] = P[4800 + t];
    S.w3[t] = P[4864 + t];
  }
  if (t == 0) {
    S.b3 = P[4928];
    mbar_init(&S.mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (t < 32) {
    tmem_alloc(&S.tbase, kTmemCols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

__device__ inline void mlp_tc_teardown(MlpSmem& S) {
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (threadIdx.x < 32) tmem_dealloc(S.tbase, kTmemCols);
}

// One tile: thread t holds sample t's (normalised) inputs x[10] and gets its
// output.  Returns false (uniformly) if an MMA did not complete in time.
__device__ inline bool mlp_tc_tile(MlpSmem& S, unsigned& phase, const float x[10], float& y) {
  const int t = threadIdx.x, warp = t >> 5;
  char* a1 = reinterpret_cast<char*>(S.A1);
  char* a2 = reinterpret_cast<char*>(S.A2);
#pragma unroll
  for (int k = 0; k < 16; ++k)
    *reinterpret_cast<__nv_bfloat16*>(a1 + kmajor_offset(t, k, 16)) = __float2bfloat16_rn(k < 10 ? x[k] : 0.f);
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  constexpr uint32_t id = idesc_bf16(128, 64);
  if (t == 0) {
    mma_bf16(S.tbase, smem_desc(S.A1, 128, 256), smem_desc(S.B1, 128, 256), id, 0);
    mma_commit(&S.mbar);
  }
  bool ok = mbar_wait(&S.mbar, phase);
  phase ^= 1u;
  if (!__syncthreads_and(ok)) return false;
  fence_after_sync();
  const unsigned lane_addr = S.tbase + ((unsigned)(warp * 32) << 16);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tmem_ld16(lane_addr + 16 * c, v);
    tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = 16 * c + q;
      *reinterpret_cast<__nv_bfloat16*>(a2 + kmajor_offset(t, j, 64)) =
          __float2bfloat16_rn(tanh_approx(v[q] + S.b1[j]));
    }
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (t == 0) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
      mma_bf16(S.tbase + 64, smem_desc(a2 + 256 * ks, 128, 1024),
               smem_desc(reinterpret_cast<char*>(S.B2) + 256 * ks, 128, 1024), id, ks > 0);
    mma_commit(&S.mbar);
  }
  ok = mbar_wait(&S.mbar, phase);
  phase ^= 1u;
  if (!__syncthreads_and(ok)) return false;
  fence_after_sync();
  float acc = S.b3;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tmem_ld16(lane_addr + 64 + 16 * c, v);
    tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = 16 * c + q;
      acc = fmaf(S.w3[j], tanh_approx(v[q] + S.b2[j]), acc);
    }
  }
  y = acc;
  return true;
}

}  // namespace tc
}  // namespace dvm

namespace dvm {
namespace tc {

// Shared memory of the tensor-core training kernel (loss and gradient of the
// 10-64-64-1 network, 128 samples per tile).  Operands (bf16, K-major):
//   A1 [128 x 16]  inputs            B1 [64 x 16]  W1
//   A2 [128 x 64]  h1                B2 [64 x 64]  W2
//   A3 [128 x 64]  d2 = dL/dz2       B3 [64 x 64]  W2^T (rows i, K = j)
//   AG [128 x 128] rows 0-63: d2^T, rows 64-127: d1^T (K = samples)
//   BG [96 x 128]  rows 0-63: h1^T, 64-79: x^T (padded), 80: ones (K = samples)
// TMEM columns: [0, 64) layer-1 pre-activations, then dL/dh1; [64, 128) layer 2;
// [128, 224) the weight-gradient accumulator D_G = AG BG^T.
struct TrainSmem {
  __nv_bfloat16 A1[128 * 16];
  __nv_bfloat16 B1[64 * 16];
  __nv_bfloat16 A2[128 * 64];
  __nv_bfloat16 B2[64 * 64];
  __nv_bfloat16 A3[128 * 64];
  __nv_bfloat16 B3[64 * 64];
  __nv_bfloat16 AG[128 * 128];
  __nv_bfloat16 BG[96 * 128];
  float b1[64], b2[64], w3[64], b3;
  float gw3[64], gb3;  // CTA sums of dL/dW3, dL/db3
  uint64_t mbar;
  unsigned tbase;
};

constexpr unsigned kTrainTmemCols = 256;

__device__ __forceinline__ void st_bf16(void* base, int off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(base) + off) = __float2bfloat16_rn(v);
}

}  // namespace tc
}  // namespace dvm
