// dvm_window.cuh -- per-source quantities of the windowed kinetic pass on
// FP32 parameters (dvm_window_kernel.cuh).  A thread owns Y consecutive
// target rows; the sources of its targets at one velocity pair (kx, kz) and
// consecutive ky form a window of source rows that slides by one row per ky
// step.  Each window slot holds the source's parameters folded with vx and
// vz, so that the Maxwellian, the deferred term and the moment-matching term
// are quadratics in vy.
#pragma once

#include "dvm_internal.cuh"

namespace dvm {

struct Slot {
  // M = exp2(c0 + c1 vy + c2 vy^2); lambda (f + nu'.m) = lambda f + a0 + a1 vy + a2 vy^2;
  // mu''.m = b0 + b1 vy + b2 vy^2 (vx and vz folded in)
  float lam, c0, c1, c2, a0, a1, a2, b0, b1, b2;
};

__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Parameters of source cell src (grouped layout, four rows per float4):
// loaded one step before they are folded, so that the loads are in flight
// while the current step computes.
struct RawSlot {
  float4 g0, g1, g2, g3;
};

__device__ __forceinline__ RawSlot load_raw(const float4* __restrict__ pg, long long nc4, int src) {
  RawSlot r;
  r.g0 = __ldg(pg + src);
  r.g1 = __ldg(pg + nc4 + src);
  r.g2 = __ldg(pg + 2 * nc4 + src);
  r.g3 = __ldg(pg + 3 * nc4 + src);
  return r;
}

// Per-cell parameters of the window pass, folded once per step from the
// parameter rows (k_window_fold): with L' = L - h |u|^2, h2_i = 2 h u_i and
// Lambda_i = lambda nu'_i the exponent of the Maxwellian at v is
//   L' + h2 . v - h |v|^2,
// and lambda nu'.m and mu''.m are linear in (1, v, |v|^2).  Groups of four:
//   3D: (lambda, L', h, h2_y) (h2_x, h2_z, Lambda_0, Lambda_x)
//       (Lambda_y, Lambda_z, Lambda_4, mu_0) (mu_x, mu_y, mu_z, mu_4)
//   2D: (lambda, L', h, h2_y) (h2_x, Lambda_0, Lambda_x, Lambda_y)
//       (Lambda_4, mu_0, mu_x, mu_y) (mu_4, 0, 0, 0)
// (index 4 is the coefficient of |v|^2).  Folding them with the fixed vx and
// vz of a velocity pair leaves quadratics in vy.
template <int D>
__device__ __forceinline__ Slot fold_slot(const RawSlot& r, float vx, float vz, float vxz2) {
  const float4 g0 = r.g0, g1 = r.g1, g2 = r.g2, g3 = r.g3;
  Slot s;
  const float h = g0.z;
  s.lam = g0.x;
  s.c2 = -h;
  s.c1 = g0.w;
  if (D == 3) {
    s.c0 = fmaf(-h, vxz2, fmaf(vz, g1.y, fmaf(vx, g1.x, g0.y)));
    s.a0 = fmaf(g2.z, vxz2, fmaf(g2.y, vz, fmaf(g1.w, vx, g1.z)));
    s.a1 = g2.x;
    s.a2 = g2.z;
    s.b0 = fmaf(g3.w, vxz2, fmaf(g3.z, vz, fmaf(g3.x, vx, g2.w)));
    s.b1 = g3.y;
    s.b2 = g3.w;
  } else {
    s.c0 = fmaf(-h, vxz2, fmaf(vx, g1.x, g0.y));
    s.a0 = fmaf(g2.x, vxz2, fmaf(g1.z, vx, g1.y));
    s.a1 = g1.w;
    s.a2 = g2.x;
    s.b0 = fmaf(g3.x, vxz2, fmaf(g2.z, vx, g2.y));
    s.b1 = g2.w;
    s.b2 = g3.x;
  }
  return s;
}

// 3D HOFKS without the learned path: the deferred term lambda nu'.m and the
// moment-matching term mu''.m enter the stored value only as their sum, so
// the window keeps one quadratic P = (Lambda + mu'').m (the moments of the
// mu''.m part come per cell from dvm_linmom.cu).  Three groups:
//   (lambda, L', h, h2_y) (h2_x, h2_z, P_0, P_x) (P_y, P_z, P_4, 0)
struct SlotP {
  // M = exp2(c0 + c1 vy + c2 vy^2); P = p0 + p1 vy + p2 vy^2
  float lam, c0, c1, c2, p0, p1, p2;
};

template <int D>
__device__ __forceinline__ SlotP fold_slot_p(const RawSlot& r, float vx, float vz, float vxz2) {
  static_assert(D == 3, "the single-quadratic form is the 3D pass's");
  const float4 g0 = r.g0, g1 = r.g1, g2 = r.g2;
  SlotP s;
  const float h = g0.z;
  s.lam = g0.x;
  s.c2 = -h;
  s.c1 = g0.w;
  s.c0 = fmaf(-h, vxz2, fmaf(vz, g1.y, fmaf(vx, g1.x, g0.y)));
  s.p0 = fmaf(g2.z, vxz2, fmaf(g2.y, vz, fmaf(g1.w, vx, g1.z)));
  s.p1 = g2.x;
  s.p2 = g2.z;
  return s;
}

template <int D>
__device__ __forceinline__ Slot load_slot(const float4* __restrict__ pg, long long nc4, int src,
                                          float vx, float vz, float vxz2) {
  return fold_slot<D>(load_raw(pg, nc4, src), vx, vz, vxz2);
}

template <int D>
__device__ __forceinline__ SlotP load_slot_p(const float4* __restrict__ pg, long long nc4, int src,
                                             float vx, float vz, float vxz2) {
  RawSlot r;
  r.g0 = __ldg(pg + src);
  r.g1 = __ldg(pg + nc4 + src);
  r.g2 = __ldg(pg + 2 * nc4 + src);
  return fold_slot_p<D>(r, vx, vz, vxz2);
}

}  // namespace dvm
