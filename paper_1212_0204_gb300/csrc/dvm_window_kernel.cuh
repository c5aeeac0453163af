// dvm_window_kernel.cuh -- the windowed kinetic pass (FP32/BF16 storage, 2D
// and 3D, periodic, integer shifts p = 1), a template over the storage type,
// dimension, scheme, staging, learned path and, optionally, compile-time
// extents.  Included by dvm_kinetic.cu (runtime extents) and
// dvm_kinetic_shapes.cu (the configured shapes).
#pragma once

#include <type_traits>

#include "dvm_internal.cuh"
#include "dvm_window.cuh"

namespace dvm {
namespace {

// ---------------------------------------------------------------------------
// Windowed kinetic pass (FP32/BF16 storage, 2D and 3D, periodic, integer
// shifts p = 1 so that delta_k = k).
//
// Warp = 32 consecutive x cells; each thread owns Y consecutive y cells of one
// z plane.  For a fixed (kz, kx) the source of target (x, y_j) at velocity ky
// is (x - kx, y_j - ky, z - kz): as ky decreases by one, every source moves
// up one row, so the Y sources of a thread form a window that slides by one
// cell per step.  The window's per-source parameters (folded with vx and vz)
// live in registers; each step loads one new source (four 16-byte loads)
// instead of Y.  The F loads of Y consecutive steps are issued together.
// Velocity moments: FP32 within a row of ky (<= 256 terms, in practice 24-32),
// FP32 across the kx of one kz plane, FP64 across planes and warps.

// 4-byte asynchronous global -> shared copy, commit and wait.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// BF16 storage: the aligned 4-byte word holding the value (cp.async copies
// 4, 8 or 16 bytes); the reader takes the half that the value's parity names.
__device__ __forceinline__ void cp_async4(float* smem, const __nv_bfloat16* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned long long a = (unsigned long long)(uintptr_t)gmem & ~3ull;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(a) : "memory");
}
// value of a staged slot: FP32 as is, BF16 from the half of the staged word
__device__ __forceinline__ float staged_value(const float* slot, int half, float*) { return *slot; }
__device__ __forceinline__ float staged_value(const float* slot, int half, __nv_bfloat16*) {
  const unsigned w = __float_as_uint(*slot);
  return __uint_as_float((half ? w & 0xffff0000u : w << 16));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// f streams through once per step: evict-first loads and stores keep the L1
// lines of the per-cell parameters (reused by neighbouring targets) resident.
template <typename TS> struct StreamT { };
template <> struct StreamT<float> {
  __device__ static float load(const float* p) { return __ldcs(p); }
  __device__ static void store(float* p, float v) { __stcs(p, v); }
};
template <> struct StreamT<__nv_bfloat16> {
  __device__ static float load(const __nv_bfloat16* p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldcs(reinterpret_cast<const unsigned short*>(p))));
  }
  __device__ static void store(__nv_bfloat16* p, float v) {
    __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v)));
  }
};

struct WinLaunch {
  int S;       // warps per CTA, each on every S-th velocity pair (kz, kx)
  int splits;  // velocity chunks across CTAs (partial-sum slices)
};

// Shape of the windowed pass per dimension, measured on GB300: warps per CTA
// (each on every S-th velocity pair; their parameter loads share L1 lines),
// resident CTAs per SM it is compiled for (register cap 65536 / (32 S MINB)),
// how many of the parameter groups of the next source row are loaded a step
// ahead of their fold (the others at fold time: more in flight costs
// registers; 3D loads all three groups of its single-quadratic form ahead),
// and the targets (consecutive y cells) per thread.  The DVM_W2_*
// / DVM_W3_* macros override them at compile time (shape sweeps).
#ifndef DVM_W2_S
#define DVM_W2_S 8
#endif
#ifndef DVM_W2_MINB
#define DVM_W2_MINB 2
#endif
#ifndef DVM_W2_EARLY
#define DVM_W2_EARLY 2
#endif
#ifndef DVM_W2_Y
#define DVM_W2_Y 4
#endif
#ifndef DVM_W3_S
#define DVM_W3_S 4
#endif
#ifndef DVM_W3_MINB
#define DVM_W3_MINB 3
#endif
#ifndef DVM_W3_EARLY
#define DVM_W3_EARLY 3
#endif
#ifndef DVM_W3_Y
#define DVM_W3_Y 4
#endif
template <int D> struct WinShape {
  static constexpr int S = DVM_W2_S, MINB = DVM_W2_MINB, EARLY = DVM_W2_EARLY, Y = DVM_W2_Y;
};
template <> struct WinShape<3> {
  static constexpr int S = DVM_W3_S, MINB = DVM_W3_MINB, EARLY = DVM_W3_EARLY, Y = DVM_W3_Y;
};
int win_warps(int d) { return d == 3 ? WinShape<3>::S : WinShape<2>::S; }
int win_y(int d) { return d == 3 ? WinShape<3>::Y : WinShape<2>::Y; }

// CTA = S warps on the same 32 x Y targets; warp s takes the velocity pairs
// pb + s, pb + s + S, ...: at any time the warps read source rows shifted by
// one column from each other, so their parameter loads share L1 lines.
// CX, CY, CZ, CV != 0: the extents N_x, N_y, N_z and the velocity count per
// dimension fixed at compile time (the configured shapes); 0: read from Geom.
template <typename TS, int D, int Y, bool HOFKS, bool ASYNC, bool LEARN, int CX = 0, int CY = 0, int CZ = 0,
          int CV = 0>
__global__ void __launch_bounds__(32 * WinShape<D>::S, WinShape<D>::MINB)
    k_kpass_window(Geom g, DevPtrs p, WinLaunch wl) {
  constexpr int NM = D + 2;
  constexpr int NA = HOFKS ? 2 * NM : NM;
  constexpr int NT = HOFKS ? 2 : 1;
  constexpr int S = WinShape<D>::S;
  constexpr int kWinT = 32 * S;
  constexpr int EARLY = WinShape<D>::EARLY;
  // 3D HOFKS without the learned path keeps one quadratic per source (SlotP)
  // and sums the new value and the Maxwellian part instead of the two parts
  // a and b; U_* and U_M follow per cell with the moments of the transported
  // mu''.m term (dvm_linmom.cu)
  constexpr bool CP = HOFKS && !LEARN && D == 3;
  using SlotT = typename std::conditional<CP, SlotP, Slot>::type;
  __shared__ int s_ox[kMaxV1], s_oy[kMaxV1], s_oz[kMaxV1];
  // dynamic: FP64 sums per (moment, target) and lane, shared by the S warps,
  // then each thread's FP32 sums of the current kz plane
  extern __shared__ double s_dyn[];
  double (*s_acc)[32] = reinterpret_cast<double (*)[32]>(s_dyn);
  float (*s_mid)[kWinT] = reinterpret_cast<float (*)[kWinT]>(s_dyn + NA * Y * 32);
  const int tid = threadIdx.x;
  const long long n1 = *p.step + 1;
  const int Nx = CX ? CX : g.nx[0], Ny = CY ? CY : g.nx[1];
  const int Nz = D == 3 ? (CZ ? CZ : g.nx[2]) : 1;
  const int nvx = CV ? CV : g.nv[0], nvy = CV ? CV : g.nv[1];
  const int nvz = D == 3 ? (CV ? CV : g.nv[2]) : 1;
  for (int t = tid; t < kMaxV1; t += kWinT) {
    if (t < nvx) s_ox[t] = wrap((long long)(g.kmin[0] + t) * n1, Nx);
    if (t < nvy) s_oy[t] = wrap((long long)(g.kmin[1] + t) * n1, Ny);
    if (D == 3 && t < nvz) s_oz[t] = wrap((long long)(g.kmin[2] + t) * n1, Nz);
  }
  for (int i = 0; i < NA * Y; ++i) s_mid[i][tid] = 0.f;
  for (int i = tid; i < NA * Y * 32; i += kWinT) s_acc[i / 32][i % 32] = 0.0;
  __syncthreads();

  const int lane = tid & 31, ws = tid >> 5;
  const int xr = blockIdx.x * 32 + lane;
  const bool xact = xr < Nx;
  const int x = xact ? xr : Nx - 1;
  const int y0 = blockIdx.y * Y;
  const int z = D == 3 ? (int)(blockIdx.z % Nz) : 0;
  const int split = D == 3 ? (int)(blockIdx.z / Nz) : (int)blockIdx.z;
  const long long nc = CX ? (long long)CX * CY * (D == 3 ? CZ : 1) : g.nc;
  const int plane = Nx * Ny;
  const float dv = (float)g.dv;
  const float4* __restrict__ pg = (const float4*)p.wprm;  // folded per cell (k_window_fold)
  TS* __restrict__ F = (TS*)p.F;
  bool tact[Y], sact[Y];
#pragma unroll
  for (int j = 0; j < Y; ++j) tact[j] = sact[j] = xact && (y0 + j < Ny);
  // learned path: flagged targets are not stored; a CTA whose targets and
  // all their sources are flagged has U_* = 0 and nothing to store, and only
  // writes its zero partial sums
  bool skip = false;
  if (LEARN) {
    int all_deep = 1;
#pragma unroll
    for (int j = 0; j < Y; ++j) {
      if (!tact[j]) continue;
      const long long cell = x + (long long)Nx * (y0 + j) + (long long)plane * z;
      sact[j] = !p.lflag[cell];
      all_deep &= p.ldeep[cell] != 0;
    }
    skip = __syncthreads_and(all_deep) != 0;
  }

  float lam_c[Y];
  if (!HOFKS) {
#pragma unroll
    for (int j = 0; j < Y; ++j) {
      const int yy = y0 + j < Ny ? y0 + j : Ny - 1;
      lam_c[j] = __ldg((const float*)p.prm + prm_at(row_lam(), x + Nx * yy + plane * z, nc));
    }
  }
  // velocity pairs (kz, kx) of this CTA (whole kz planes in 3D, a multiple of
  // S pairs); this warp takes every S-th one
  const int npairs = nvx * (D == 3 ? nvz : 1);
  const int per = npairs / wl.splits;
  const int pb = split * per, pe = pb + per;
  // first window row: y0 - (kmin_y + nvy - 1), wrapped once per thread
  int sy_first = (y0 - (g.kmin[1] + nvy - 1)) % Ny;
  if (sy_first < 0) sy_first += Ny;
  const long long kystep = (long long)nvx * nc;  // F offset between consecutive ky

  // FP32 storage: the F values of a block of Y velocities x Y targets go
  // through shared memory by cp.async, one block ahead of the arithmetic
  // (more loads in flight than registers allow; no register holds them)
  // (BF16 with N_x even: a value's word half is the parity of its x piece)
  float* s_fb = reinterpret_cast<float*>(s_mid + NA * Y);  // [2][Y][Y][kWinT]
  int stage = 0;
  auto issue = [&](int base_i, int kb_i, int st) {
    const int pr_i = base_i + ws;
    const int kx_i = pr_i % nvx;
    const int kz_i = D == 3 ? pr_i / nvx : 0;
    int qx_i = x - s_ox[kx_i];
    if (qx_i < 0) qx_i += Nx;
    int qz_i = 0;
    if (D == 3) {
      qz_i = z - s_oz[kz_i];
      if (qz_i < 0) qz_i += Nz;
    }
    const TS* Fb_i = F + ((long long)kx_i + (long long)nvx * nvy * kz_i) * nc + qx_i + plane * qz_i;
    // every address is a valid one (x clamped, rows wrapped): inactive
    // targets copy a value nobody reads instead of taking a predicate
    int rr[Y];
    bool nowrap = true;
#pragma unroll
    for (int jj = 0; jj < Y; ++jj) {
      int r = y0 - s_oy[kb_i - jj];
      if (r < 0) r += Ny;
      rr[jj] = r;
      nowrap = nowrap && r + Y <= Ny;
    }
    float* dst = s_fb + st * Y * Y * kWinT + tid;
    if (nowrap) {  // no periodic wrap among the rows of the block (CTA-uniform)
#pragma unroll
      for (int jj = 0; jj < Y; ++jj) {
        const TS* Fr = Fb_i + (long long)(kb_i - jj) * kystep + rr[jj] * Nx;
#pragma unroll
        for (int j = 0; j < Y; ++j) cp_async4(dst + (jj * Y + j) * kWinT, Fr + j * Nx);
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < Y; ++jj) {
        const TS* Fk = Fb_i + (long long)(kb_i - jj) * kystep;
        int r = rr[jj];
#pragma unroll
        for (int j = 0; j < Y; ++j) {
          cp_async4(dst + (jj * Y + j) * kWinT, Fk + r * Nx);
          if (++r == Ny) r = 0;
        }
      }
    }
  };
  if (ASYNC && !skip && pb < pe) {
    issue(pb, nvy - 1, 0);
    cp_async_commit();
  }
  for (int base = skip ? pe : pb; base < pe; base += S) {
    const int pr = base + ws;
    const int kx = pr % nvx;
    const int kz = D == 3 ? pr / nvx : 0;
    const int kxg = g.kmin[0] + kx, kzg = D == 3 ? g.kmin[2] + kz : 0;
    const float vx = kxg * dv, vz = kzg * dv;
    const float vxz2 = fmaf(vx, vx, vz * vz);
    int sx = (x - kxg) % Nx;
    if (sx < 0) sx += Nx;
    int sz = 0, qz = 0;
    if (D == 3) {
      sz = (z - kzg) % Nz;
      if (sz < 0) sz += Nz;
      qz = z - s_oz[kz];
      if (qz < 0) qz += Nz;
    }
    int qx = x - s_ox[kx];
    if (qx < 0) qx += Nx;
    const int src_base = sx + plane * sz;
    const int dst_base = qx + plane * qz;
    TS* __restrict__ Fb = F + ((long long)kx + (long long)nvx * nvy * kz) * nc + dst_base;
    // window: slot i holds source row (sy_first + i), wrapped
    SlotT win[Y];
    int rnext = sy_first;
#pragma unroll
    for (int i = 0; i < Y; ++i) {
      if constexpr (CP) win[i] = load_slot_p<D>(pg, nc, src_base + Nx * rnext, vx, vz, vxz2);
      else win[i] = load_slot<D>(pg, nc, src_base + Nx * rnext, vx, vz, vxz2);
      if (++rnext == Ny) rnext = 0;
    }
    float in0[NT][Y], in1[NT][Y], in2[NT][Y];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int j = 0; j < Y; ++j) in0[t][j] = in1[t][j] = in2[t][j] = 0.f;
    for (int kb = nvy - 1; kb >= 0; kb -= Y) {
      float fv[ASYNC ? 1 : Y][Y];
      if constexpr (ASYNC) {
        // this block's values landed in shared memory (prefetched one block
        // ahead); queue the next block (or the next pair's first) meanwhile;
        // its stage was last read one block ago (an empty group past the end
        // keeps the group count uniform)
        if (kb - Y >= 0) issue(base, kb - Y, stage ^ 1);
        else if (base + S < pe) issue(base + S, nvy - 1, stage ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        // the F loads of Y steps first: Y*Y independent loads in flight
#pragma unroll
        for (int jj = 0; jj < Y; ++jj) {
          const int ky = kb - jj;
          int r = y0 - s_oy[ky];
          if (r < 0) r += Ny;
          const TS* Fk = Fb + (long long)ky * kystep;
          if (r + Y <= Ny) {  // no periodic wrap among the Y rows (warp-uniform)
            const TS* Fr = Fk + r * Nx;
#pragma unroll
            for (int j = 0; j < Y; ++j) fv[jj][j] = tact[j] ? StreamT<TS>::load(Fr + j * Nx) : 0.f;
          } else {
#pragma unroll
            for (int j = 0; j < Y; ++j) {
              fv[jj][j] = tact[j] ? StreamT<TS>::load(Fk + r * Nx) : 0.f;
              if (++r == Ny) r = 0;
            }
          }
        }
      }
      // rows of the Y steps' targets; one CTA-uniform test per block picks
      // the body without periodic wraps (a single basic block over the Y
      // steps, so the parameter loads of one step overlap the next ones)
      bool nowrap = true;
#pragma unroll
      for (int jj = 0; jj < Y; ++jj) {
        int r = y0 - s_oy[kb - jj];
        if (r < 0) r += Ny;
        nowrap = nowrap && r + Y <= Ny;
      }
      auto steps = [&](auto fast) {
#pragma unroll
        for (int jj = 0; jj < Y; ++jj) {
          const int ky = kb - jj;
          // the source row that enters the window after this step: its loads
          // are issued before this step's arithmetic (after the last step of
          // a pair the row is loaded and folded but not used)
          RawSlot raw;
          const int src_next = src_base + Nx * rnext;
          raw.g0 = __ldg(pg + src_next);
          if (EARLY > 1) raw.g1 = __ldg(pg + nc + src_next);
          if (EARLY > 2) raw.g2 = __ldg(pg + 2 * nc + src_next);
          if (EARLY > 3 && !CP) raw.g3 = __ldg(pg + 3 * nc + src_next);
          float fj[Y];
#pragma unroll
          for (int j = 0; j < Y; ++j)
            fj[j] = ASYNC ? staged_value(&s_fb[((stage * Y + jj) * Y + j) * kWinT + tid], qx & 1, (TS*)nullptr)
                          : fv[ASYNC ? 0 : jj][j];
          const float vy = (g.kmin[1] + ky) * dv;
          const float vy2 = vy * vy;
          float fn[Y];
#pragma unroll
          for (int j = 0; j < Y; ++j) {
            const SlotT& sl = win[(jj + j) % Y];
            const float M = ex2_ftz(fmaf(sl.c2, vy2, fmaf(sl.c1, vy, sl.c0)));
            if constexpr (CP) {
              // new value lambda f + P + M; sums of it and of M
              const float P = fmaf(sl.p2, vy2, fmaf(sl.p1, vy, sl.p0));
              const float fv = fmaf(sl.lam, fj[j], P) + M;
              fn[j] = fv;
              in0[0][j] += fv;
              in1[0][j] = fmaf(fv, vy, in1[0][j]);
              in2[0][j] = fmaf(fv, vy2, in2[0][j]);
              in0[1][j] += M;
              in1[1][j] = fmaf(M, vy, in1[1][j]);
              in2[1][j] = fmaf(M, vy2, in2[1][j]);
            } else if constexpr (HOFKS) {
              const float lm = fmaf(sl.b2, vy2, fmaf(sl.b1, vy, sl.b0));
              const float a = fmaf(sl.lam, fj[j], fmaf(sl.a2, vy2, fmaf(sl.a1, vy, sl.a0)));
              const float b = M + lm;  // T((1 - lambda) E^n)
              fn[j] = a + b;           // a = T(lambda f^n)
              in0[0][j] += a;
              in1[0][j] = fmaf(a, vy, in1[0][j]);
              in2[0][j] = fmaf(a, vy2, in2[0][j]);
              in0[NT - 1][j] += b;
              in1[NT - 1][j] = fmaf(b, vy, in1[NT - 1][j]);
              in2[NT - 1][j] = fmaf(b, vy2, in2[NT - 1][j]);
            } else {
              const float lm = fmaf(sl.b2, vy2, fmaf(sl.b1, vy, sl.b0));
              const float fs = fj[j] + M + lm;  // transported f
              fn[j] = lam_c[j] * fs;            // its lambda part; the rest is deferred
              in0[0][j] += fs;
              in1[0][j] = fmaf(fs, vy, in1[0][j]);
              in2[0][j] = fmaf(fs, vy2, in2[0][j]);
            }
          }
          TS* Fk = Fb + ky * kystep;
          int r = y0 - s_oy[ky];
          if (r < 0) r += Ny;
          if constexpr (decltype(fast)::value) {
            TS* Fr = Fk + r * Nx;
#pragma unroll
            for (int j = 0; j < Y; ++j)
              if (sact[j]) StreamT<TS>::store(Fr + j * Nx, fn[j]);
          } else {
#pragma unroll
            for (int j = 0; j < Y; ++j) {
              if (sact[j]) StreamT<TS>::store(Fk + r * Nx, fn[j]);
              if (++r == Ny) r = 0;
            }
          }
          // slide: the slot just left by target 0 takes the next source row
          if (EARLY <= 1) raw.g1 = __ldg(pg + nc + src_next);
          if (EARLY <= 2) raw.g2 = __ldg(pg + 2 * nc + src_next);
          if (EARLY <= 3 && !CP) raw.g3 = __ldg(pg + 3 * nc + src_next);
          if constexpr (CP) win[jj % Y] = fold_slot_p<D>(raw, vx, vz, vxz2);
          else win[jj % Y] = fold_slot<D>(raw, vx, vz, vxz2);
          if (++rnext == Ny) rnext = 0;
        }
      };
      if (nowrap) steps(std::true_type{});
      else steps(std::false_type{});
      if (ASYNC) stage ^= 1;
    }
    // fold the row sums into the plane sums: m = (1, vx, vy, [vz], |v|^2/2)
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int o = t * NM;
#pragma unroll
      for (int j = 0; j < Y; ++j) {
        const float s0 = in0[t][j];
        s_mid[(o + 0) * Y + j][tid] += s0;
        s_mid[(o + 1) * Y + j][tid] = fmaf(vx, s0, s_mid[(o + 1) * Y + j][tid]);
        s_mid[(o + 2) * Y + j][tid] += in1[t][j];
        if (D == 3) s_mid[(o + 3) * Y + j][tid] = fmaf(vz, s0, s_mid[(o + 3) * Y + j][tid]);
        s_mid[(o + D + 1) * Y + j][tid] += 0.5f * fmaf(vxz2, s0, in2[t][j]);
      }
    }
    // plane finished (same round for all S warps): their FP32 plane sums
    // into the shared FP64 accumulators
    if ((base + S) % nvx == 0 || base + S >= pe) {
      __syncthreads();
      for (int i = tid; i < NA * Y * 32; i += kWinT) {
        const int e = i / 32, l = i % 32;
        // the S warps' plane sums in FP32, then one FP64 add (GB300's FP64
        // rate is 1/64 of FP32: one conversion and one add per element)
        float v = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < S; ++w2) v += s_mid[e][l + 32 * w2];
        s_acc[e][l] += (double)v;
      }
      __syncthreads();
#pragma unroll
      for (int a = 0; a < NA * Y; ++a) s_mid[a][tid] = 0.f;
    }
  }
  if (ASYNC) cp_async_wait<0>();
  // this split's partial sums
  __syncthreads();
  for (int i = tid; i < NA * Y * 32; i += kWinT) {
    const int e = i / 32, l = i % 32;
    const int a = e / Y, j = e % Y;
    const int xx = blockIdx.x * 32 + l;
    if (xx >= Nx || y0 + j >= Ny) continue;
    const long long cell = xx + (long long)Nx * (y0 + j) + (long long)plane * z;
    // combined form: the first part holds the sums of the new value, so
    // U_* - (its mu''.m part) is that minus the Maxwellian part's sums
    const double v = CP && a < NM ? s_acc[e][l] - s_acc[e + NM * Y][l] : s_acc[e][l];
    p.acc[((long long)split * 2 * NM + a) * nc + cell] = v;
  }
}

constexpr size_t window_smem(int d, bool hofks, bool async) {
  const size_t t = 32 * (d == 3 ? WinShape<3>::S : WinShape<2>::S);
  const size_t y = d == 3 ? WinShape<3>::Y : WinShape<2>::Y;
  return (size_t)(hofks ? 2 : 1) * (d + 2) * y * (32 * sizeof(double) + t * sizeof(float)) +
         (async ? (size_t)2 * y * y * t * sizeof(float) : 0);
}

}  // namespace
}  // namespace dvm
