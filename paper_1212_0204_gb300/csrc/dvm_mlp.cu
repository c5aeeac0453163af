// dvm_mlp.cu -- the regime network on its own: inference over device
// samples, mean-squared-error gradient and Adam training (dvm_mlp_* in
// dvm.h).  FP32 kernels on the CUDA cores; the BF16 forward pass runs on the
// tensor cores (tcgen05, building blocks in dvm_tc.cuh).
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "dvm_internal.cuh"
#include "dvm_mlp.cuh"
#include "dvm_tc.cuh"

using namespace dvm;

struct dvm_mlp {
  int precision = DVM_F32;
  cudaStream_t stream = nullptr;
  float* P = nullptr;      // FP32 master parameters
  float* m = nullptr;      // Adam first moment
  float* v = nullptr;      // Adam second moment
  double* grad = nullptr;  // gradient of the current batch
  double* loss = nullptr;  // 1: sum of squared errors of the current batch
  int* perm = nullptr;     // epoch order
  long long perm_cap = 0;
  long long t = 0;         // Adam steps taken
  int* status = nullptr;   // device: tensor-core wait timed out
  bool set = false;
  std::string err;
};

namespace dvm {
namespace {

constexpr int kFwdBlock = 128;

__global__ void __launch_bounds__(kFwdBlock) k_mlp_forward_f32(const float* __restrict__ P, long long n,
                                                               const float* __restrict__ X,
                                                               float* __restrict__ y) {
  __shared__ __align__(16) float sP[kNP + 3];
  for (int i = threadIdx.x; i < kNP; i += kFwdBlock) sP[i] = P[i];
  __syncthreads();
  const long long s = blockIdx.x * (long long)kFwdBlock + threadIdx.x;
  if (s >= n) return;
  float x[kNIn];
#pragma unroll
  for (int i = 0; i < kNIn; ++i) x[i] = X[s * kNIn + i];
  y[s] = mlp_forward_f32(sP, x);
}

// Loss and gradient of a batch, FP32 arithmetic, one CTA per 64 samples.
// Activations live in shared memory with a padded row stride (65) so that
// a warp reading one column of 32 samples hits 32 banks.  The CTA's gradient
// is summed over its samples in FP32 and added to the FP64 total.
constexpr int kGS = 64;            // samples per CTA
constexpr int kGThreads = 256;
constexpr int kLD = kNH + 1;       // padded row stride of activations
constexpr int kGradSmemFloats = kNP + 4 + kGS * kNIn + 4 * kGS * kLD + 2 * kGS;

__global__ void __launch_bounds__(kGThreads) k_mlp_grad_f32(const float* __restrict__ P, long long n,
                                                            const float* __restrict__ X,
                                                            const float* __restrict__ T,
                                                            const int* __restrict__ idx,
                                                            long long first, long long count,
                                                            float scale, double* __restrict__ grad,
                                                            double* __restrict__ loss) {
  extern __shared__ __align__(16) float sm[];
  float* sP = sm;                           // kNP
  float* sX = sP + kNP + 4;                 // [kGS][kNIn]
  float* H1 = sX + kGS * kNIn;              // [kGS][kLD]
  float* H2 = H1 + kGS * kLD;
  float* D2 = H2 + kGS * kLD;
  float* D1 = D2 + kGS * kLD;
  float* dy = D1 + kGS * kLD;               // kGS
  float* ok = dy + kGS;                     // kGS: 1 for a real sample
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long b0 = blockIdx.x * (long long)kGS;
  for (int i = tid; i < kNP; i += kGThreads) sP[i] = P[i];
  for (int i = tid; i < kGS * kNIn; i += kGThreads) {
    const int s = i / kNIn, f = i % kNIn;
    const long long j = b0 + s;
    float v = 0.f;
    if (j < count) {
      const long long r = idx ? idx[first + j] : first + j;
      v = X[r * kNIn + f];
    }
    sX[i] = v;
  }
  __syncthreads();
  const float* W1 = sP + kOffW1;
  const float* b1 = sP + kOffB1;
  const float* W2 = sP + kOffW2;
  const float* b2 = sP + kOffB2;
  const float* W3 = sP + kOffW3;
  // H1[s][j] = tanh(b1_j + W1_j . x_s): lane -> s (two halves), warp -> j
  for (int o = tid; o < kGS * kNH; o += kGThreads) {
    const int s = o % kGS, j = o / kGS;
    float a = b1[j];
#pragma unroll
    for (int i = 0; i < kNIn; ++i) a = fmaf(W1[j * kNIn + i], sX[s * kNIn + i], a);
    H1[s * kLD + j] = tanhf(a);
  }
  __syncthreads();
  for (int o = tid; o < kGS * kNH; o += kGThreads) {
    const int s = o % kGS, j = o / kGS;
    float a = b2[j];
#pragma unroll 16
    for (int i = 0; i < kNH; ++i) a = fmaf(W2[j * kNH + i], H1[s * kLD + i], a);
    H2[s * kLD + j] = tanhf(a);
  }
  __syncthreads();
  // y_s, error, dL/dy (warp w handles samples w, w + 8, ...)
  float lsum = 0.f;
  for (int s = warp; s < kGS; s += kGThreads / 32) {
    float a = W3[lane] * H2[s * kLD + lane] + W3[lane + 32] * H2[s * kLD + lane + 32];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) {
      const long long j = b0 + s;
      const bool real = j < count;
      float e = 0.f;
      if (real) {
        const long long r = idx ? idx[first + j] : first + j;
        e = a + sP[kOffB3] - T[r];
      }
      dy[s] = real ? 2.f * e * scale : 0.f;
      ok[s] = real ? 1.f : 0.f;
      lsum += e * e;
    }
  }
  if (lane == 0) atomicAdd(loss, (double)lsum);
  __syncthreads();
  for (int o = tid; o < kGS * kNH; o += kGThreads) {
    const int s = o % kGS, j = o / kGS;
    const float h = H2[s * kLD + j];
    D2[s * kLD + j] = dy[s] * W3[j] * (1.f - h * h);
  }
  __syncthreads();
  // D1[s][i] = (1 - H1^2) sum_j D2[s][j] W2[j][i]
  for (int o = tid; o < kGS * kNH; o += kGThreads) {
    const int s = o % kGS, i = o / kGS;
    float a = 0.f;
#pragma unroll 16
    for (int j = 0; j < kNH; ++j) a = fmaf(D2[s * kLD + j], W2[j * kNH + i], a);
    const float h = H1[s * kLD + i];
    D1[s * kLD + i] = a * (1.f - h * h);
  }
  __syncthreads();
  // parameter gradients: sums over the CTA's samples
  for (int o = tid; o < kNP; o += kGThreads) {
    float a = 0.f;
    if (o < kOffB1) {  // W1[j][i]
      const int j = o / kNIn, i = o % kNIn;
      for (int s = 0; s < kGS; ++s) a = fmaf(D1[s * kLD + j], sX[s * kNIn + i], a);
    } else if (o < kOffW2) {  // b1
      const int j = o - kOffB1;
      for (int s = 0; s < kGS; ++s) a += D1[s * kLD + j];
    } else if (o < kOffB2) {  // W2[j][i]
      const int j = (o - kOffW2) / kNH, i = (o - kOffW2) % kNH;
      for (int s = 0; s < kGS; ++s) a = fmaf(D2[s * kLD + j], H1[s * kLD + i], a);
    } else if (o < kOffW3) {  // b2
      const int j = o - kOffB2;
      for (int s = 0; s < kGS; ++s) a += D2[s * kLD + j];
    } else if (o < kOffB3) {  // W3
      const int j = o - kOffW3;
      for (int s = 0; s < kGS; ++s) a = fmaf(dy[s], H2[s * kLD + j], a);
    } else {  // b3
      for (int s = 0; s < kGS; ++s) a += dy[s];
    }
    atomicAdd(&grad[o], (double)a);
  }
}

// BF16 tensor-core forward pass (tcgen05, FP32 accumulate in TMEM), one
// 128-sample tile at a time per CTA.
__global__ void __launch_bounds__(tc::kTcThreads) k_mlp_forward_tc(const float* __restrict__ P, long long n,
                                                                   const float* __restrict__ X,
                                                                   float* __restrict__ y, int* status) {
  __shared__ __align__(1024) tc::MlpSmem S;
  tc::mlp_tc_setup(S, P);
  unsigned phase = 0;
  const long long ntiles = (n + 127) / 128;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long s = tile * 128 + threadIdx.x;
    float x[kNIn];
#pragma unroll
    for (int i = 0; i < kNIn; ++i) x[i] = s < n ? X[s * kNIn + i] : 0.f;
    float out = 0.f;
    if (!tc::mlp_tc_tile(S, phase, x, out)) {
      if (threadIdx.x == 0) atomicCAS(status, 0, DVM_ERR_TIMEOUT);
      break;
    }
    if (s < n) y[s] = out;
  }
  tc::mlp_tc_teardown(S);
}


// Loss and gradient on the tensor cores (BF16 operands, FP32 accumulation):
// CTAs walk 128-sample tiles; the weight gradient of all its tiles stays in
// TMEM (D_G += AG BG^T per tile) and is added to the FP64 total once.
__global__ void __launch_bounds__(tc::kTcThreads) k_mlp_grad_tc(const float* __restrict__ P,
                                                                const float* __restrict__ X,
                                                                const float* __restrict__ T,
                                                                const int* __restrict__ idx,
                                                                long long first, long long count,
                                                                float scale, double* __restrict__ grad,
                                                                double* __restrict__ loss, int* status) {
  extern __shared__ __align__(1024) unsigned char s_raw[];
  tc::TrainSmem& S = *reinterpret_cast<tc::TrainSmem*>(s_raw);
  const int t = threadIdx.x, warp = t >> 5;
  using tc::kmajor_offset;
  using tc::st_bf16;
  // ---- setup: weights in operand layout, biases, accumulators, mbarrier, TMEM
  for (int i = t; i < 64 * 16; i += tc::kTcThreads) {
    const int j = i / 16, k = i % 16;
    st_bf16(S.B1, kmajor_offset(j, k, 16), k < 10 ? P[kOffW1 + j * 10 + k] : 0.f);
  }
  for (int i = t; i < 64 * 64; i += tc::kTcThreads) {
    const int j = i / 64, k = i % 64;
    const float w = P[kOffW2 + i];        // W2[j][k]
    st_bf16(S.B2, kmajor_offset(j, k, 64), w);
    st_bf16(S.B3, kmajor_offset(k, j, 64), w);  // W2^T: row k, column j
  }
  // BG rows 80..95: ones (row 80) and zeros, set once
  for (int i = t; i < 16 * 128; i += tc::kTcThreads) {
    const int r = 80 + i / 128, s = i % 128;
    st_bf16(S.BG, kmajor_offset(r, s, 128), r == 80 ? 1.f : 0.f);
  }
  if (t < 64) {
    S.b1[t] = P[kOffB1 + t];
    S.b2[t] = P[kOffB2 + t];
    S.w3[t] = P[kOffW3 + t];
    S.gw3[t] = 0.f;
  }
  if (t == 0) {
    S.b3 = P[kOffB3];
    S.gb3 = 0.f;
    tc::mbar_init(&S.mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (t < 32) {
    tc::tmem_alloc(&S.tbase, tc::kTrainTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const unsigned lane_addr = S.tbase + ((unsigned)(warp * 32) << 16);
  constexpr uint32_t id64 = tc::idesc_bf16(128, 64), id96 = tc::idesc_bf16(128, 96);
  unsigned phase = 0;
  int ntile = 0;
  bool ok = true;
  float lsum = 0.f;
  const long long ntiles = (count + 127) / 128;
  auto sync_mma = [&]() {  // operands written -> visible to the tensor cores
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  auto wait_mma = [&]() -> bool {
    const bool w = tc::mbar_wait(&S.mbar, phase);
    phase ^= 1u;
    const bool all = __syncthreads_and(w) != 0;
    tc::fence_after_sync();
    return all;
  };
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++ntile) {
    const long long j = tile * 128 + t;
    const bool real = j < count;
    const long long r = real ? (idx ? idx[first + j] : first + j) : 0;
    float x[kNIn];
#pragma unroll
    for (int i = 0; i < kNIn; ++i) x[i] = real ? X[r * kNIn + i] : 0.f;
    const float target = real ? T[r] : 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float v = k < 10 ? x[k] : 0.f;
      st_bf16(S.A1, kmajor_offset(t, k, 16), v);
      st_bf16(S.BG, kmajor_offset(64 + k, t, 128), v);  // x^T
    }
    sync_mma();
    if (t == 0) {
      tc::mma_bf16(S.tbase, tc::smem_desc(S.A1, 128, 256), tc::smem_desc(S.B1, 128, 256), id64, 0);
      tc::mma_commit(&S.mbar);
    }
    if (!(ok = wait_mma())) break;
    float h1[64];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tc::tmem_ld16(lane_addr + 16 * c, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = 16 * c + q;
        h1[i] = tc::tanh_approx(v[q] + S.b1[i]);
        st_bf16(S.A2, kmajor_offset(t, i, 64), h1[i]);
        st_bf16(S.BG, kmajor_offset(i, t, 128), h1[i]);  // h1^T
      }
    }
    sync_mma();
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc::mma_bf16(S.tbase + 64, tc::smem_desc(reinterpret_cast<char*>(S.A2) + 256 * ks, 128, 1024),
                     tc::smem_desc(reinterpret_cast<char*>(S.B2) + 256 * ks, 128, 1024), id64, ks > 0);
      tc::mma_commit(&S.mbar);
    }
    if (!(ok = wait_mma())) break;
    // output, error, dL/dy; d2 = dy W3 (1 - h2^2); dW3 and db3 sums
    float h2[64];
    float y = S.b3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tc::tmem_ld16(lane_addr + 64 + 16 * c, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = 16 * c + q;
        h2[i] = tc::tanh_approx(v[q] + S.b2[i]);
        y = fmaf(S.w3[i], h2[i], y);
      }
    }
    const float e = real ? y - target : 0.f;
    const float dy = 2.f * e * scale;
    lsum = fmaf(e, e, lsum);
    const int lane = t & 31;
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      const float d2 = dy * S.w3[i] * (1.f - h2[i] * h2[i]);
      st_bf16(S.A3, kmajor_offset(t, i, 64), d2);
      st_bf16(S.AG, kmajor_offset(i, t, 128), d2);  // d2^T
      float g = dy * h2[i];  // dL/dW3_i of this sample, summed over the warp
      for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
      if (lane == 0) atomicAdd(&S.gw3[i], g);
    }
    {
      float g = dy;
      for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
      if (lane == 0) atomicAdd(&S.gb3, g);
    }
    sync_mma();
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc::mma_bf16(S.tbase, tc::smem_desc(reinterpret_cast<char*>(S.A3) + 256 * ks, 128, 1024),
                     tc::smem_desc(reinterpret_cast<char*>(S.B3) + 256 * ks, 128, 1024), id64, ks > 0);
      tc::mma_commit(&S.mbar);
    }
    if (!(ok = wait_mma())) break;
    // d1 = dL/dh1 (1 - h1^2) into AG rows 64..127
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tc::tmem_ld16(lane_addr + 16 * c, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = 16 * c + q;
        st_bf16(S.AG, kmajor_offset(64 + i, t, 128), v[q] * (1.f - h1[i] * h1[i]));
      }
    }
    sync_mma();
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        tc::mma_bf16(S.tbase + 128, tc::smem_desc(reinterpret_cast<char*>(S.AG) + 256 * ks, 128, 2048),
                     tc::smem_desc(reinterpret_cast<char*>(S.BG) + 256 * ks, 128, 2048), id96,
                     (ntile > 0 || ks > 0) ? 1 : 0);
      tc::mma_commit(&S.mbar);
    }
    // AG and BG are rewritten by the next tile: wait for this product
    if (!(ok = wait_mma())) break;
  }
  if (!ok) {
    if (t == 0) atomicCAS(status, 0, DVM_ERR_TIMEOUT);
  } else if (ntile > 0) {
    // D_G rows: lane r < 64 -> (dW2[r][0..63], db2[r] at column 80);
    //           lane 64 + i -> (dW1[i][0..9] at columns 64..73, db1[i] at 80)
    float v[16];
    if (warp < 2) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tc::tmem_ld16(lane_addr + 128 + 16 * c, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 16; ++q) atomicAdd(&grad[kOffW2 + t * 64 + 16 * c + q], (double)v[q]);
      }
      tc::tmem_ld16(lane_addr + 128 + 80, v);
      tc::tmem_ld_wait();
      atomicAdd(&grad[kOffB2 + t], (double)v[0]);
    } else {
      const int i = t - 64;
      tc::tmem_ld16(lane_addr + 128 + 64, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int k = 0; k < 10; ++k) atomicAdd(&grad[kOffW1 + i * 10 + k], (double)v[k]);
      tc::tmem_ld16(lane_addr + 128 + 80, v);
      tc::tmem_ld_wait();
      atomicAdd(&grad[kOffB1 + i], (double)v[0]);
    }
    __syncthreads();
    if (t < 64) atomicAdd(&grad[kOffW3 + t], (double)S.gw3[t]);
    if (t == 0) atomicAdd(&grad[kOffB3], (double)S.gb3);
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0) atomicAdd(loss, (double)lsum);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (t < 32) tc::tmem_dealloc(S.tbase, tc::kTrainTmemCols);
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const double* __restrict__ grad, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  const float gr = (float)grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gr;
  const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

unsigned long long splitmix(unsigned long long& s) {
  unsigned long long z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

int mfail(dvm_mlp* m, int code, const std::string& msg) {
  m->err = msg;
  return code;
}

int mcheck(dvm_mlp* m, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return 0;
  return mfail(m, DVM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// gradient (and summed squared error) of samples first .. first + count of
// the order idx (or of X itself) into m->grad / m->loss, which the caller zeroes
void launch_grad(dvm_mlp* m, long long n, const float* X, const float* T, const int* idx,
                 long long first, long long count, float scale) {
  cudaStream_t s = m->stream;
  if (m->precision == DVM_BF16S) {
    const long long tiles = (count + 127) / 128;
    const unsigned nb = (unsigned)(tiles < 152 ? tiles : 152);  // ~114 KB shared: one CTA per SM
    k_mlp_grad_tc<<<nb, tc::kTcThreads, sizeof(tc::TrainSmem), s>>>(m->P, X, T, idx, first, count, scale,
                                                                    m->grad, m->loss, m->status);
  } else {
    const unsigned nb = (unsigned)((count + kGS - 1) / kGS);
    k_mlp_grad_f32<<<nb, kGThreads, kGradSmemFloats * sizeof(float), s>>>(m->P, n, X, T, idx, first,
                                                                           count, scale, m->grad, m->loss);
  }
}

int grad_batch(dvm_mlp* m, long long n, const float* X, const float* T, const int* idx,
               long long first, long long count, float scale) {
  cudaStream_t s = m->stream;
  int rc = mcheck(m, cudaMemsetAsync(m->grad, 0, sizeof(double) * (kNP + 1), s), "memset");
  if (rc) return rc;
  launch_grad(m, n, X, T, idx, first, count, scale);
  return mcheck(m, cudaGetLastError(), "gradient launch");
}

int check_status(dvm_mlp* m) {
  if (m->precision != DVM_BF16S) return 0;
  int st = 0;
  if (mcheck(m, cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost), "status")) return DVM_ERR_CUDA;
  return st ? mfail(m, st, "tensor-core kernel did not complete") : 0;
}

}  // namespace
}  // namespace dvm

extern "C" {

int dvm_mlp_create(int precision, void* cuda_stream, dvm_mlp** out) {
  if (!out) return DVM_ERR_ARG;
  *out = nullptr;
  if (precision != DVM_F32 && precision != DVM_BF16S) return DVM_ERR_ARG;
  dvm_mlp* m = new dvm_mlp();
  m->precision = precision;
  m->stream = (cudaStream_t)cuda_stream;
  char* b = nullptr;
  const size_t pb = 256 * ((sizeof(float) * kNP + 255) / 256);
  const size_t gb = 256 * ((sizeof(double) * (kNP + 2) + 255) / 256);
  if (cudaMalloc((void**)&b, 3 * pb + gb) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return DVM_ERR_OOM;
  }
  m->P = (float*)b;
  m->m = (float*)(b + pb);
  m->v = (float*)(b + 2 * pb);
  m->grad = (double*)(b + 3 * pb);
  m->loss = m->grad + kNP;
  m->status = (int*)(m->loss + 1);
  cudaFuncSetAttribute(k_mlp_grad_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(kGradSmemFloats * sizeof(float)));
  cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(tc::TrainSmem));
  if (cudaMemsetAsync(b, 0, 3 * pb + gb, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b);
    delete m;
    return DVM_ERR_CUDA;
  }
  *out = m;
  return 0;
}

void dvm_mlp_destroy(dvm_mlp* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  else cudaDeviceSynchronize();
  if (m->P) cudaFree(m->P);
  if (m->perm) cudaFree(m->perm);
  delete m;
}

int dvm_mlp_set_params(dvm_mlp* m, const float* P) {
  if (!m || !P) return DVM_ERR_ARG;
  cudaStream_t s = m->stream;
  int rc = 0;
  rc |= mcheck(m, cudaMemcpyAsync(m->P, P, sizeof(float) * kNP, cudaMemcpyHostToDevice, s), "copy");
  rc |= mcheck(m, cudaMemsetAsync(m->m, 0, sizeof(float) * kNP, s), "memset");
  rc |= mcheck(m, cudaMemsetAsync(m->v, 0, sizeof(float) * kNP, s), "memset");
  rc |= mcheck(m, cudaStreamSynchronize(s), "sync");
  if (rc) return DVM_ERR_CUDA;
  m->t = 0;
  m->set = true;
  return 0;
}

int dvm_mlp_get_params(dvm_mlp* m, float* P) {
  if (!m || !P) return DVM_ERR_ARG;
  int rc = mcheck(m, cudaMemcpyAsync(P, m->P, sizeof(float) * kNP, cudaMemcpyDeviceToHost, m->stream), "copy");
  rc |= mcheck(m, cudaStreamSynchronize(m->stream), "sync");
  return rc ? DVM_ERR_CUDA : 0;
}

int dvm_mlp_forward(dvm_mlp* m, long long n, const float* X, float* y) {
  if (!m || n < 0 || (n > 0 && (!X || !y))) return DVM_ERR_ARG;
  if (!m->set) return mfail(m, DVM_ERR_STATE, "parameters not set");
  if (n == 0) return 0;
  if (m->precision == DVM_BF16S) {
    const long long tiles = (n + 127) / 128;
    const unsigned grid = (unsigned)(tiles < 152 * 4 ? tiles : 152 * 4);
    k_mlp_forward_tc<<<grid, tc::kTcThreads, 0, m->stream>>>(m->P, n, X, y, m->status);
  } else {
    k_mlp_forward_f32<<<(unsigned)((n + kFwdBlock - 1) / kFwdBlock), kFwdBlock, 0, m->stream>>>(m->P, n, X, y);
  }
  int rc = mcheck(m, cudaGetLastError(), "forward launch");
  if (!rc) rc = mcheck(m, cudaStreamSynchronize(m->stream), "sync");
  if (rc) return DVM_ERR_CUDA;
  int st = 0;
  if (m->precision == DVM_BF16S) {
    rc = mcheck(m, cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost), "status");
    if (rc) return DVM_ERR_CUDA;
    if (st) return mfail(m, st, "tensor-core forward did not complete");
  }
  return 0;
}

int dvm_mlp_loss_grad(dvm_mlp* m, long long n, const float* X, const float* t, double* grad,
                      double* loss) {
  if (!m || n < 1 || !X || !t || !grad) return DVM_ERR_ARG;
  if (!m->set) return mfail(m, DVM_ERR_STATE, "parameters not set");
  int rc = grad_batch(m, n, X, t, nullptr, 0, n, 1.f / (float)n);
  if (rc) return rc;
  double l = 0.0;
  rc |= mcheck(m, cudaMemcpyAsync(grad, m->grad, sizeof(double) * kNP, cudaMemcpyDeviceToDevice, m->stream), "copy");
  rc |= mcheck(m, cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream), "copy");
  rc |= mcheck(m, cudaStreamSynchronize(m->stream), "sync");
  if (rc) return DVM_ERR_CUDA;
  if ((rc = check_status(m))) return rc;
  if (loss) *loss = l / (double)n;
  return 0;
}

int dvm_mlp_train(dvm_mlp* m, long long n, const float* X, const float* t,
                  const dvm_train_config* cfg, double* loss) {
  if (!m || n < 1 || !X || !t || !cfg || cfg->epochs < 0 || cfg->batch < 1) return DVM_ERR_ARG;
  if (!m->set) return mfail(m, DVM_ERR_STATE, "parameters not set");
  if (n > 0x7fffffffLL) return mfail(m, DVM_ERR_ARG, "too many samples");
  cudaStream_t s = m->stream;
  if (m->perm_cap < n) {
    if (m->perm) cudaFree(m->perm);
    m->perm = nullptr;
    if (cudaMalloc((void**)&m->perm, sizeof(int) * (size_t)n) != cudaSuccess) {
      cudaGetLastError();
      m->perm_cap = 0;
      return mfail(m, DVM_ERR_OOM, "epoch order");
    }
    m->perm_cap = n;
  }
  std::vector<int> perm((size_t)n);
  unsigned long long seed = cfg->seed;
  double last = 0.0;
  int rc = 0;
  for (int e = 0; e < cfg->epochs; ++e) {
    for (long long i = 0; i < n; ++i) perm[(size_t)i] = (int)i;
    for (long long i = n - 1; i > 0; --i) {
      const long long j = (long long)(splitmix(seed) % (unsigned long long)(i + 1));
      const int tmp = perm[(size_t)i];
      perm[(size_t)i] = perm[(size_t)j];
      perm[(size_t)j] = tmp;
    }
    if ((rc = mcheck(m, cudaMemcpyAsync(m->perm, perm.data(), sizeof(int) * (size_t)n,
                                        cudaMemcpyHostToDevice, s), "copy"))) return rc;
    if ((rc = mcheck(m, cudaMemsetAsync(m->loss, 0, sizeof(double), s), "memset"))) return rc;
    for (long long b = 0; b < n; b += cfg->batch) {
      const long long cnt = (n - b) < cfg->batch ? (n - b) : cfg->batch;
      // the loss accumulates over the epoch: keep it out of the reset
      if ((rc = mcheck(m, cudaMemsetAsync(m->grad, 0, sizeof(double) * kNP, s), "memset"))) return rc;
      launch_grad(m, n, X, t, m->perm, b, cnt, 1.f / (float)cnt);
      ++m->t;
      const float c1 = 1.f / (1.f - powf(cfg->beta1, (float)m->t));
      const float c2 = 1.f / (1.f - powf(cfg->beta2, (float)m->t));
      k_adam<<<(kNP + 255) / 256, 256, 0, s>>>(m->P, m->m, m->v, m->grad, cfg->lr, cfg->beta1,
                                               cfg->beta2, cfg->eps, c1, c2);
    }
    if ((rc = mcheck(m, cudaGetLastError(), "training launch"))) return rc;
    double l = 0.0;
    if ((rc = mcheck(m, cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "copy"))) return rc;
    if ((rc = mcheck(m, cudaStreamSynchronize(s), "sync"))) return rc;
    if ((rc = check_status(m))) return rc;
    last = l / (double)n;
  }
  if (loss) *loss = last;
  return 0;
}

}  // extern "C"
