// dvm_kinetic.cu -- the kinetic pass: the one sweep over the whole phase
// space per time step.  For every target cell c and velocity k it
//   * finds the piece now covering c (exact transport, Section 4.2) and the
//     cell s that piece covered at t^n, by integer offsets only;
//   * reads the stored value once, adds the deferred term of cell s, and
//     relaxes it (FKS: Eq. relaxdvm; HOFKS: R then T of Section 4.3.1);
//   * accumulates the velocity moments of the cell (Eq. DM, Eq. UK);
//   * writes the new value back into the same piece (in place).
// One read and one write of f per phase-space point.
#include <math.h>

#include <cmath>
#include <stdlib.h>

#include "dvm_internal.cuh"
#include "dvm_window.cuh"
#include "dvm_window_kernel.cuh"

namespace dvm {
namespace {

constexpr int kThreads = 256;

// DVM_GENERIC_PASS=1 forces the generic kinetic pass (for comparison runs).
bool getenv_generic() {
  const char* e = getenv("DVM_GENERIC_PASS");
  return e && e[0] == '1';
}

template <typename TC> __device__ inline TC fexp2(TC x);
template <> __device__ inline float fexp2<float>(float x) { return exp2f(x); }
template <> __device__ inline double fexp2<double>(double x) { return exp2(x); }

// Generic kinetic pass: one thread per target cell, a chunk of velocities per
// blockIdx.y, moment partial sums per chunk.  Per-cell parameters of the
// source cells are read through the L1 cache.
template <typename TS, typename TC, int D, bool HOFKS>
__global__ void __launch_bounds__(kThreads) k_kpass_generic(Geom g, DevPtrs p) {
  __shared__ int s_slot[D][kMaxV1];   // o_i(k, n+1) mod N_i
  __shared__ int s_delta[D][kMaxV1];  // o_i(k, n+1) - o_i(k, n)
  __shared__ TC s_v[D][kMaxV1];
  const long long n = *p.step;
  for (int t = threadIdx.x; t < D * kMaxV1; t += blockDim.x) {
    const int i = t / kMaxV1, kk = t % kMaxV1;
    if (kk < g.nv[i]) {
      const long long k = g.kmin[i] + kk;
      const long long o1 = transport_offset(k, n + 1, g.p), o0 = transport_offset(k, n, g.p);
      s_slot[i][kk] = wrap(o1, g.nx[i]);
      s_delta[i][kk] = (int)(o1 - o0);
      s_v[i][kk] = (TC)((double)k * g.dv);
    }
  }
  __syncthreads();
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  const long long nc = g.nc;
  int x[3];
  x[0] = (int)(c % g.nx[0]);
  x[1] = D > 1 ? (int)((c / g.nx[0]) % g.nx[1]) : 0;
  x[2] = D > 2 ? (int)(c / ((long long)g.nx[0] * g.nx[1])) : 0;

  const long long kb = blockIdx.y * g.nvel / g.nsplit;
  const long long ke = (blockIdx.y + 1) * g.nvel / g.nsplit;
  // a flagged target's pieces are E by definition after the step: not stored
  const bool store = !(g.learn && p.lflag[c]);
  int kx = (int)(kb % g.nv[0]);
  int ky = D > 1 ? (int)((kb / g.nv[0]) % g.nv[1]) : 0;
  int kz = D > 2 ? (int)(kb / ((long long)g.nv[0] * g.nv[1])) : 0;

  const TC* prm = (const TC*)p.prm;
  TS* F = (TS*)p.F;
  const TS* G = (const TS*)p.ghost;
  const TC lam_c = prm[prm_at(row_lam(), c, nc)];

  constexpr int NM = D + 2;
  constexpr int NACC = HOFKS ? 2 * NM : NM;
  double acc[NACC];
  TC racc[NACC];
  for (int j = 0; j < NACC; ++j) acc[j] = 0.0, racc[j] = TC(0);

  for (long long k = kb; k < ke; ++k) {
    const int kk[3] = {kx, ky, kz};
    int s[3] = {0, 0, 0}, q[3] = {0, 0, 0};
    bool clamped = false;
    TC v[3];
    TC vv = TC(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const int N = g.nx[i];
      int t = x[i] - s_delta[i][kk[i]];
      if (g.bc[i] == DVM_BC_PERIODIC) {
        t = t < 0 ? t + N : (t >= N ? t - N : t);
        if (t < 0 || t >= N) t = wrap(t, N);
      } else if (t < 0 || t >= N) {
        t = t < 0 ? 0 : N - 1;
        clamped = true;
      }
      s[i] = t;
      int r = x[i] - s_slot[i][kk[i]];
      q[i] = r < 0 ? r + N : r;
      v[i] = s_v[i][kk[i]];
      vv += v[i] * v[i];
    }
    vv *= TC(0.5);
    const long long src = s[0] + (long long)g.nx[0] * (s[1] + (long long)g.nx[1] * s[2]);
    const long long slot = q[0] + (long long)g.nx[0] * (q[1] + (long long)g.nx[1] * q[2]);
    TC fv;
    if (!clamped) {
      fv = StoreT<TS>::load(F + k * nc + slot);
    } else if (g.ghost_mode == 1) {
      fv = StoreT<TS>::load(G + 2 * k + (s[0] == 0 ? 0 : 1));
    } else {
      int qs[3] = {0, 0, 0};
#pragma unroll
      for (int i = 0; i < D; ++i)
        qs[i] = wrap((long long)s[i] - s_slot[i][kk[i]] + s_delta[i][kk[i]], g.nx[i]);
      fv = StoreT<TS>::load(G + k * nc + qs[0] + (long long)g.nx[0] * (qs[1] + (long long)g.nx[1] * qs[2]));
    }
    // parameters of the source cell; the Maxwellian (Eq. M) from its
    // separable factors in the FP64 build (k_gauss_tables), else one exp2
    TC M;
    if constexpr (sizeof(TC) == 8) {
      M = p.gtab[src];
      int off = 1;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        M *= p.gtab[(long long)(off + kk[i]) * nc + src];
        off += g.nv[i];
      }
    } else {
      TC qq = TC(0);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const TC du = v[i] - prm[prm_at(row_u(i), src, nc)];
        qq += du * du;
      }
      M = fexp2<TC>(prm[prm_at(row_L(), src, nc)] - prm[prm_at(row_h(D), src, nc)] * qq);
    }
    TC lin_mu = prm[prm_at(row_mu(D, 0), src, nc)] + prm[prm_at(row_mu(D, D + 1), src, nc)] * (vv + vv);
#pragma unroll
    for (int i = 0; i < D; ++i) lin_mu += prm[prm_at(row_mu(D, 1 + i), src, nc)] * v[i];
    TC fnew;
    if (HOFKS) {
      TC lin_nu = prm[prm_at(row_nu(D, 0), src, nc)] + prm[prm_at(row_nu(D, D + 1), src, nc)] * (vv + vv);
#pragma unroll
      for (int i = 0; i < D; ++i) lin_nu += prm[prm_at(row_nu(D, 1 + i), src, nc)] * v[i];
      const TC a = prm[prm_at(row_lam(), src, nc)] * (fv + lin_nu);  // T(lambda f^n)
      const TC b = M + lin_mu;                                   // T((1-lambda) E^n)
      fnew = a + b;
      racc[0] += a;
      racc[NM] += b;
#pragma unroll
      for (int i = 0; i < D; ++i) racc[1 + i] += a * v[i], racc[NM + 1 + i] += b * v[i];
      racc[D + 1] += a * vv;
      racc[NM + D + 1] += b * vv;
    } else {
      const TC fs = fv + M + lin_mu;  // transported f
      fnew = lam_c * fs;              // its lambda part; the rest is deferred
      racc[0] += fs;
#pragma unroll
      for (int i = 0; i < D; ++i) racc[1 + i] += fs * v[i];
      racc[D + 1] += fs * vv;
    }
    if (store) StoreT<TS>::store(F + k * nc + slot, fnew);
    // next velocity (x fastest); flush the short compute-type sums per row
    if (++kx == g.nv[0]) {
      kx = 0;
#pragma unroll
      for (int j = 0; j < NACC; ++j) acc[j] += (double)racc[j], racc[j] = TC(0);
      if (D > 1 && ++ky == g.nv[1]) {
        ky = 0;
        if (D > 2) ++kz;
      }
    }
  }
  double* out = p.acc + (long long)blockIdx.y * 2 * NM * nc + c;
#pragma unroll
  for (int j = 0; j < NACC; ++j) out[j * nc] = acc[j] + (double)racc[j];
}

// FP64 build: the separable factors of every cell's Maxwellian (Eq. M),
// 2^L and exp2(-h (v_k - u_i)^2) per dimension i and velocity index k, from
// the parameters the kinetic pass is about to use (the Gaussian of |v - u|^2
// is the product of its per-dimension factors): the pass then forms M with
// d multiplications instead of an FP64 exp2 per phase-space point.
template <int D>
__global__ void __launch_bounds__(256) k_gauss_tables(Geom g, DevPtrs p) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nc = g.nc;
  if (c >= nc) return;
  const double* prm = (const double*)p.prm;
  const double h = prm[prm_at(row_h(D), c, nc)];
  p.gtab[c] = exp2(prm[prm_at(row_L(), c, nc)]);
  long long row = 1;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const double u = prm[prm_at(row_u(i), c, nc)];
    for (int k = 0; k < g.nv[i]; ++k, ++row) {
      const double du = (double)(g.kmin[i] + k) * g.dv - u;
      p.gtab[row * nc + c] = exp2(-h * (du * du));
    }
  }
}

// One thread per cell: the parameter rows folded into the window layout of
// dvm_window.cuh (fold_slot).
template <int D>
__global__ void __launch_bounds__(256) k_window_fold(Geom g, DevPtrs p) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nc = g.nc;
  if (c >= nc) return;
  const float4* __restrict__ pg = (const float4*)p.prm;
  float r[16];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v = __ldg(pg + q * nc + c);
    r[4 * q] = v.x, r[4 * q + 1] = v.y, r[4 * q + 2] = v.z, r[4 * q + 3] = v.w;
  }
  const float lam = r[row_lam()], L = r[row_L()], h = r[row_h(D)];
  const float ux = r[row_u(0)], uy = r[row_u(1)], uz = D == 3 ? r[row_u(2)] : 0.f;
  const float u2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
  float Lam[5], mu[5];
#pragma unroll
  for (int i = 0; i < D + 2; ++i) {
    Lam[i] = lam * r[row_nu(D, i)];
    mu[i] = r[row_mu(D, i)];
  }
  float4 o[4];
  o[0] = make_float4(lam, fmaf(-h, u2, L), h, 2.f * h * uy);
  if (D == 3) {
    o[1] = make_float4(2.f * h * ux, 2.f * h * uz, Lam[0], Lam[1]);
    o[2] = make_float4(Lam[2], Lam[3], Lam[4], mu[0]);
    o[3] = make_float4(mu[1], mu[2], mu[3], mu[4]);
  } else {
    o[1] = make_float4(2.f * h * ux, Lam[0], Lam[1], Lam[2]);
    o[2] = make_float4(Lam[3], mu[0], mu[1], mu[2]);
    o[3] = make_float4(mu[3], 0.f, 0.f, 0.f);
  }
  float4* __restrict__ wg = (float4*)p.wprm;
#pragma unroll
  for (int q = 0; q < 4; ++q) wg[q * nc + c] = o[q];
}

// 3D HOFKS without the learned path: the same rows with the deferred and the
// moment-matching quadratics summed, P = lambda nu' + mu'' (SlotP layout of
// dvm_window.cuh).
__global__ void __launch_bounds__(256) k_window_fold_p(Geom g, DevPtrs p) {
  constexpr int D = 3;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nc = g.nc;
  if (c >= nc) return;
  const float4* __restrict__ pg = (const float4*)p.prm;
  float r[16];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v = __ldg(pg + q * nc + c);
    r[4 * q] = v.x, r[4 * q + 1] = v.y, r[4 * q + 2] = v.z, r[4 * q + 3] = v.w;
  }
  const float lam = r[row_lam()], L = r[row_L()], h = r[row_h(D)];
  const float ux = r[row_u(0)], uy = r[row_u(1)], uz = r[row_u(2)];
  const float u2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
  float P[5];
#pragma unroll
  for (int i = 0; i < D + 2; ++i) P[i] = fmaf(lam, r[row_nu(D, i)], r[row_mu(D, i)]);
  float4 o[3];
  o[0] = make_float4(lam, fmaf(-h, u2, L), h, 2.f * h * uy);
  o[1] = make_float4(2.f * h * ux, 2.f * h * uz, P[0], P[1]);
  o[2] = make_float4(P[2], P[3], P[4], 0.f);
  float4* __restrict__ wg = (float4*)p.wprm;
#pragma unroll
  for (int q = 0; q < 3; ++q) wg[q * nc + c] = o[q];
}


bool window_eligible(const Geom& g) {
  if (g.d < 2 || g.precision == DVM_F64 || g.p != 1) return false;
  for (int i = 0; i < g.d; ++i)
    if (g.bc[i] != DVM_BC_PERIODIC) return false;
  // 32-bit cell indices; rows wrap with one subtraction; the S warps of a
  // CTA end every kz plane in the same round
  const int Y = win_y(g.d);
  return g.nv[1] % Y == 0 && g.nv[0] % win_warps(g.d) == 0 && g.nx[1] >= Y && g.nc < (1LL << 31);
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

// Velocity splits across CTAs (slices of the kz planes in 3D, of the nvx / S
// groups in 2D).  Among the divisors c <= 4 that leave a CTA at least 2^16
// updates, the one with the fewest CTA waves per unit of work,
// ceil(tiles c / R) / c with R the resident CTAs, so that the last wave is
// nearly full; ties go to the larger c (finer load balance).
WinLaunch window_shape(const Geom& g) {
  if (tile3_shape(g)) {
    // the 3D tile kernel (32 x 16 targets per CTA, 3 CTAs per SM): its larger
    // tiles make the last wave's fill matter more, and each split adds a pass
    // of FP64 partial sums (written here, read by the end-of-step kernel,
    // 160 B per cell against 8 N_v of f); the divisor c of N_v1 (<= 12) with
    // the smallest ceil(waves) / waves x (1 + 20 c / N_v) (96^3: 6, 64^3: 8)
    const long long tiles = (long long)(g.nx[0] / 32) * (g.nx[1] / 16) * g.nx[2];
    const double resident = (double)sm_count() * 3;
    int sp = 1;
    double best = 1e30;
    for (int c = 1; c <= 12 && c <= g.nv[2]; ++c) {
      if (g.nv[2] % c || (c > 1 && 512LL * g.nvel / c < (1LL << 16))) continue;
      const double waves = (double)(tiles * c) / resident;
      const double cost = std::ceil(waves) / waves * (1.0 + 20.0 * c / (double)g.nvel);
      if (cost < best) { best = cost; sp = c; }
    }
    WinLaunch wl;
    wl.S = win_warps(g.d);
    wl.splits = sp;
    return wl;
  }
  const int Y = win_y(g.d);
  const long long tiles = ((g.nx[0] + 31) / 32) * ((g.nx[1] + Y - 1) / Y) * g.nx[2];
  const long long resident = (long long)sm_count() * (g.d == 3 ? WinShape<3>::MINB : WinShape<2>::MINB);
  const long long cta_updates = 32LL * Y * g.nvel;
  const int units = g.d == 3 ? g.nv[2] : g.nv[0] / win_warps(g.d);
  int sp = 1;
  double best = 1e30;
  for (int c = 1; c <= 4 && c <= units; ++c) {
    if (units % c || (c > 1 && cta_updates / c < (1LL << 16))) continue;
    const double waves = (double)((tiles * c + resident - 1) / resident) / c;
    if (waves <= best) { best = waves; sp = c; }
  }
  WinLaunch wl;
  wl.S = win_warps(g.d);
  wl.splits = sp;
  return wl;
}


// FP32 staging of the F loads through shared memory: on by default (with 8
// warps per CTA it measures faster in 2D and 3D; DVM_WIN_ASYNC=0/1 overrides).
bool window_async(int d) {
  const char* e = getenv("DVM_WIN_ASYNC");
  if (e && (e[0] == '0' || e[0] == '1')) return e[0] == '1';
  (void)d;
  return true;
}

template <typename TS, int D, bool HO, bool AS>
void launch_window_a(const Geom& g, const DevPtrs& p, const WinLaunch& wl, cudaStream_t s, bool prepare) {
  if constexpr (!std::is_same<TS, double>::value && HO && AS) {
    // a configured shape: the kernel with compile-time extents (FP32; BF16
    // staged, which the caller selects for an even N_x only)
    const bool fixed = launch_window_fixed(g, p, wl.splits, s, prepare);
    if (fixed && !prepare) return;
  }
  constexpr size_t sm = window_smem(D, HO, AS);
  if (prepare) {
    cudaFuncSetAttribute(k_kpass_window<TS, D, WinShape<D>::Y, HO, AS, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_kpass_window<TS, D, WinShape<D>::Y, HO, AS, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return;
  }
  constexpr int Y = WinShape<D>::Y;
  dim3 grid((unsigned)((g.nx[0] + 31) / 32), (unsigned)((g.nx[1] + Y - 1) / Y),
            (unsigned)(g.nx[2] * wl.splits));
  constexpr int T = 32 * WinShape<D>::S;
  if (g.learn) k_kpass_window<TS, D, Y, HO, AS, true><<<grid, T, sm, s>>>(g, p, wl);
  else k_kpass_window<TS, D, Y, HO, AS, false><<<grid, T, sm, s>>>(g, p, wl);
}

template <typename TS, int D, bool HO>
void launch_window_t(const Geom& g, const DevPtrs& p, const WinLaunch& wl, cudaStream_t s, bool prepare) {
  // staged f loads: FP32, and BF16 when N_x is even (a value's half of its
  // staged 4-byte word is then the parity of its x piece)
  if (prepare) launch_window_a<TS, D, HO, true>(g, p, wl, s, true);
  else if (window_async(D) && (sizeof(TS) == 4 || g.nx[0] % 2 == 0))
    return launch_window_a<TS, D, HO, true>(g, p, wl, s, false);
  launch_window_a<TS, D, HO, false>(g, p, wl, s, prepare);
}

template <typename TS>
void launch_window(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare = false) {
  const WinLaunch wl = window_shape(g);
  const bool ho = g.scheme != DVM_FKS;
  if (g.d == 2) {
    if (ho) launch_window_t<TS, 2, true>(g, p, wl, s, prepare);
    else launch_window_t<TS, 2, false>(g, p, wl, s, prepare);
  } else {
    if (ho) launch_window_t<TS, 3, true>(g, p, wl, s, prepare);
    else launch_window_t<TS, 3, false>(g, p, wl, s, prepare);
  }
}

template <typename TS, typename TC>
void launch_generic(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  dim3 grid((unsigned)((g.nc + kThreads - 1) / kThreads), (unsigned)g.nsplit);
  const bool ho = g.scheme != DVM_FKS;
#define DVM_KP(DD)                                                              \
  if (ho) k_kpass_generic<TS, TC, DD, true><<<grid, kThreads, 0, s>>>(g, p);    \
  else k_kpass_generic<TS, TC, DD, false><<<grid, kThreads, 0, s>>>(g, p);
  if (g.d == 1) { DVM_KP(1) } else if (g.d == 2) { DVM_KP(2) } else { DVM_KP(3) }
#undef DVM_KP
}

}  // namespace

// Velocity chunks: enough blocks for several waves on 152 SMs, at least 16
// velocities per chunk.
int kinetic_pass_splits(const Geom& g) {
  if (window_eligible(g)) return window_shape(g).splits;
  const long long blocks = (g.nc + kThreads - 1) / kThreads;
  const long long want = 152LL * 8;
  long long s = (want + blocks - 1) / blocks;
  const long long maxs = g.nvel / 16 > 0 ? g.nvel / 16 : 1;
  if (s > maxs) s = maxs;
  if (s > 64) s = 64;
  if (s < 1) s = 1;
  return (int)s;
}

// Kernel attributes that must be set before the first launch (outside any
// stream capture): dynamic shared memory of the windowed pass.
void kinetic_pass_prepare(const Geom& g) {
  if (!window_eligible(g)) return;
  if (g.lin_slice) linear_moments_prepare(g);
  DevPtrs none{};
  if (g.precision == DVM_F32) launch_window<float>(g, none, nullptr, true);
  else launch_window<__nv_bfloat16>(g, none, nullptr, true);
}

// The windowed pass (it skips CTAs whose targets are all deep in the learned
// path).
bool kinetic_is_windowed(const Geom& g) {
  return window_eligible(g) && !getenv_generic();
}

int launch_kinetic_pass(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  if (kinetic_is_windowed(g)) {
    const unsigned nb = (unsigned)((g.nc + 255) / 256);
    if (g.d == 3 && g.scheme != DVM_FKS && !g.learn) {
      k_window_fold_p<<<nb, 256, 0, s>>>(g, p);
    } else if (g.d == 2) {
      k_window_fold<2><<<nb, 256, 0, s>>>(g, p);
    } else {
      k_window_fold<3><<<nb, 256, 0, s>>>(g, p);
    }
    if (g.precision == DVM_F32) launch_window<float>(g, p, s);
    else launch_window<__nv_bfloat16>(g, p, s);
    return 2;
  }
  if (g.precision == DVM_F64) {
    const unsigned nb = (unsigned)((g.nc + 255) / 256);
    if (g.d == 1) k_gauss_tables<1><<<nb, 256, 0, s>>>(g, p);
    else if (g.d == 2) k_gauss_tables<2><<<nb, 256, 0, s>>>(g, p);
    else k_gauss_tables<3><<<nb, 256, 0, s>>>(g, p);
    launch_generic<double, double>(g, p, s);
    return 2;
  }
  if (g.precision == DVM_F32) launch_generic<float, float>(g, p, s);
  else launch_generic<__nv_bfloat16, float>(g, p, s);
  return 1;
}

}  // namespace dvm
