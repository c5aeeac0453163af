// dvm_learn.cuh -- device state and launchers of the learned regime path
// (shared by dvm_api.cu and dvm_learn.cu; never installed).
#pragma once

#include "dvm_internal.cuh"

namespace dvm {

// Device buffers of the learned path (all owned by the handle).
struct LearnDev {
  unsigned char* flag;       // nc: flags of the current / last step
  unsigned char* flag_prev;  // nc: flags of the step before
  unsigned char* given;      // nc: caller flags (GIVEN mode)
  unsigned char* veto;       // nc: cells kept unflagged
  unsigned char* deep;       // nc: flagged with every source of the step flagged
  unsigned char* tmp;        // nc: scratch of the deep filter
  float* pred;               // nc: network output of the step
  float* tauf;               // nc: tau (FP32, inf allowed)
  double* lw;                // nc: -log2(1 - lambda)
  double* invw;              // nc: 1 / (1 - lambda)
  float* P;                  // DVM_MLP_NPARAM network parameters (FP32)
  __nv_bfloat16* Pb;         // BF16 copy (tensor-core inference)
  float* norm;               // 2 x 10: input shift, scale
  int* mat_list;             // nc: cells to write back as E
  unsigned int* mat_count;   // 1
  unsigned long long* cnt;   // counters, see kCnt*
  double* err;               // [0] sum |pred - true|, [1] max |pred - true|, [2] max true
  long long* check_cells;    // kMaxCheck
  float* check_out;          // kMaxCheck
};

constexpr int kMaxCheck = 65536;
enum { kCntFlagged = 0, kCntMaterialised = 1, kCntChecked = 2, kCntFailed = 3, kCntVetoed = 4,
       kCntN = 8 };

// per step, before the Euler part (all on one stream)
void learn_launch_flags(const Geom& g, const DevPtrs& p, const LearnDev& L, int mode,
                        int mlp_precision, float thr, cudaStream_t s);
void learn_launch_apply(const Geom& g, const DevPtrs& p, const LearnDev& L, cudaStream_t s);
void learn_launch_deep(const Geom& g, const LearnDev& L, cudaStream_t s);
void learn_launch_materialise(const Geom& g, const DevPtrs& p, const LearnDev& L, cudaStream_t s);
// after the Euler part and the ghost snapshot, before the kinetic pass
void learn_launch_check(const Geom& g, const DevPtrs& p, const LearnDev& L, int ncheck,
                        bool explicit_cells, float thr, int radius, unsigned long long seed,
                        bool mlp, cudaStream_t s);
// read-back helpers
void learn_launch_features(const Geom& g, const DevPtrs& p, const LearnDev& L, float* out,
                           cudaStream_t s);
void learn_launch_noneq(const Geom& g, const DevPtrs& p, float* out, cudaStream_t s);
void learn_launch_flush(const Geom& g, const DevPtrs& p, const LearnDev& L, cudaStream_t s);
void learn_prepare(const Geom& g);
bool kinetic_is_windowed(const Geom& g);

}  // namespace dvm
