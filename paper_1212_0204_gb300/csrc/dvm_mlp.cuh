// dvm_mlp.cuh -- device helpers of the regime network (10-64-64-1, tanh
// hidden layers, linear output), shared by the learned path and the
// training kernels.
#pragma once

#include "dvm_internal.cuh"

namespace dvm {

constexpr int kNIn = DVM_NFEAT, kNH = DVM_MLP_HIDDEN, kNP = DVM_MLP_NPARAM;
// offsets in the packed parameter vector
constexpr int kOffW1 = 0, kOffB1 = kNH * kNIn, kOffW2 = kOffB1 + kNH, kOffB2 = kOffW2 + kNH * kNH,
              kOffW3 = kOffB2 + kNH, kOffB3 = kOffW3 + kNH;

// FP32 forward pass of the 10-64-64-1 tanh network, parameters in shared
// memory (every thread reads the same address: broadcast).
__device__ inline float mlp_forward_f32(const float* __restrict__ sP, const float x[kNIn]) {
  const float* W1 = sP;
  const float* b1 = W1 + kNH * kNIn;
  const float* W2 = b1 + kNH;
  const float* b2 = W2 + kNH * kNH;
  const float* W3 = b2 + kNH;
  const float b3 = W3[kNH];
  float h1[kNH];
#pragma unroll
  for (int j = 0; j < kNH; ++j) {
    float s = b1[j];
#pragma unroll
    for (int i = 0; i < kNIn; ++i) s = fmaf(W1[j * kNIn + i], x[i], s);
    h1[j] = tanhf(s);
  }
  float y = b3;
#pragma unroll 4
  for (int j = 0; j < kNH; ++j) {
    const float4* w = reinterpret_cast<const float4*>(W2 + j * kNH);
    float s = b2[j];
#pragma unroll
    for (int i = 0; i < kNH / 4; ++i) {
      const float4 q = w[i];
      s = fmaf(q.x, h1[4 * i], s);
      s = fmaf(q.y, h1[4 * i + 1], s);
      s = fmaf(q.z, h1[4 * i + 2], s);
      s = fmaf(q.w, h1[4 * i + 3], s);
    }
    y = fmaf(W3[j], tanhf(s), y);
  }
  return y;
}

}  // namespace dvm
