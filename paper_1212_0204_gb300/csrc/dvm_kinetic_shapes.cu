// dvm_kinetic_shapes.cu -- the kinetic pass compiled with the grid extents
// and velocity counts of the configured workloads fixed at compile time (2D
// 128^2, 256^2, 512^2 x 32^2; 3D 32^3, 64^3, 96^3 x 24^3): the index and
// address arithmetic then works on constants (on GB300 about a quarter of the
// per-thread window kernel's instructions).  2D FP32 HOFKS (also with the
// learned path) and BF16 storage (2D 256^2 / 512^2, 3D 64^3 / 96^3) run the
// per-thread window kernel (dvm_window_kernel.cuh); 3D FP32 HOFKS runs the
// kernel whose CTA shares each pair's folded source rows (dvm_tile_kernel.cuh;
// also at 32^3 x 8^3, the shape of its oracle test).  Every other
// configuration runs the window kernel with the extents read at run time
// (dvm_kinetic.cu).
#include <stdlib.h>

#include "dvm_tile_kernel.cuh"

namespace dvm {
namespace {

// 3D FP32 HOFKS without the learned path: the kernel with the CTA's source
// rows folded once into shared memory (dvm_tile_kernel.cuh)
template <int CX, int CY, int CZ, int CV>
bool try_tile3(const Geom& g, const DevPtrs& p, int splits, cudaStream_t s, bool prepare) {
  if (g.nx[0] != CX || g.nx[1] != CY || g.nx[2] != CZ) return false;
  if (g.nv[0] != CV || g.nv[1] != CV || g.nv[2] != CV) return false;
  constexpr size_t sm = tile_smem(CV);
  auto* k = k_kpass_tile3<float, CX, CY, CZ, CV>;
  if (prepare) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return true;
  }
  if (g.learn) return false;
  const dim3 grid((unsigned)(CX / 32), (unsigned)(CY / kTileTY), (unsigned)(CZ * splits));
  k<<<grid, 32 * kTileW, sm, s>>>(g, p, splits);
  return true;
}

template <int D, int CX, int CY, int CZ, int CV, bool LE, typename TS = float>
bool try_shape(const Geom& g, const DevPtrs& p, int splits, cudaStream_t s, bool prepare) {
  if (g.nx[0] != CX || g.nx[1] != CY || (D == 3 && g.nx[2] != CZ)) return false;
  if (g.nv[0] != CV || g.nv[1] != CV || (D == 3 && g.nv[2] != CV)) return false;
  if (!prepare && (g.learn != 0) != LE) return false;
  // (BF16 pieces are staged as aligned 4-byte words: N_x even)
  static_assert(sizeof(TS) == 4 || CX % 2 == 0, "BF16 staging needs an even N_x");
  constexpr size_t sm = window_smem(D, true, true);
  constexpr int Y = WinShape<D>::Y;
  auto* k = k_kpass_window<TS, D, Y, true, true, LE, CX, CY, CZ, CV>;
  if (prepare) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return true;
  }
  WinLaunch wl;
  wl.S = WinShape<D>::S;
  wl.splits = splits;
  const dim3 grid((unsigned)((CX + 31) / 32), (unsigned)((CY + Y - 1) / Y),
                  (unsigned)((D == 3 ? CZ : 1) * splits));
  k<<<grid, 32 * WinShape<D>::S, sm, s>>>(g, p, wl);
  return true;
}

}  // namespace

// 3D FP32 HOFKS at a shape with a tile kernel (the splits are chosen for it)
bool tile3_shape(const Geom& g) {
  if (g.d != 3 || g.precision != DVM_F32 || g.scheme == DVM_FKS) return false;
  if (g.nx[0] != g.nx[1] || g.nx[1] != g.nx[2] || g.nv[0] != g.nv[1] || g.nv[1] != g.nv[2]) return false;
  const int n = g.nx[0], v = g.nv[0];
  return (v == 24 && (n == 32 || n == 64 || n == 96)) || (v == 8 && n == 32);
}

// DVM_FIXED_SHAPES=0 runs the runtime-extent kernel for every shape (for
// comparison runs and the test that both give the same result).
bool launch_window_fixed(const Geom& g, const DevPtrs& p, int splits, cudaStream_t s, bool prepare) {
  if (g.precision == DVM_F64 || g.scheme == DVM_FKS) return false;
  const char* e = getenv("DVM_FIXED_SHAPES");
  if (e && e[0] == '0' && !prepare) return false;
  if (g.precision == DVM_BF16S) {
    // BF16 storage: the 2D 256^2 / 512^2 and 3D 64^3 / 96^3 shapes, no learned path
    if (g.learn) return false;
    if (g.d == 2)
      return try_shape<2, 256, 256, 1, 32, false, __nv_bfloat16>(g, p, splits, s, prepare) ||
             try_shape<2, 512, 512, 1, 32, false, __nv_bfloat16>(g, p, splits, s, prepare);
    if (g.d == 3)
      return try_shape<3, 64, 64, 64, 24, false, __nv_bfloat16>(g, p, splits, s, prepare) ||
             try_shape<3, 96, 96, 96, 24, false, __nv_bfloat16>(g, p, splits, s, prepare);
    return false;
  }
  if (g.d == 2) {
    // with and without the learned path (both prepared at creation)
    bool hit = false;
    hit |= try_shape<2, 256, 256, 1, 32, false>(g, p, splits, s, prepare) ||
           try_shape<2, 512, 512, 1, 32, false>(g, p, splits, s, prepare) ||
           try_shape<2, 128, 128, 1, 32, false>(g, p, splits, s, prepare);
    if (hit && !prepare) return true;
    hit |= try_shape<2, 256, 256, 1, 32, true>(g, p, splits, s, prepare) ||
           try_shape<2, 512, 512, 1, 32, true>(g, p, splits, s, prepare) ||
           try_shape<2, 128, 128, 1, 32, true>(g, p, splits, s, prepare);
    return hit;
  }
  if (g.d == 3)  // (without the learned path: try_tile3 declines it)
    return try_tile3<64, 64, 64, 24>(g, p, splits, s, prepare) || try_tile3<96, 96, 96, 24>(g, p, splits, s, prepare) ||
           try_tile3<32, 32, 32, 24>(g, p, splits, s, prepare) || try_tile3<32, 32, 32, 8>(g, p, splits, s, prepare);
  return false;
}

}  // namespace dvm
