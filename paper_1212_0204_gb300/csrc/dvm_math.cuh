// dvm_math.cuh -- device math shared by the libdvm translation units:
// primitive variables, separable Gaussian sums of the discrete Maxwellian,
// the Euler flux and the van Leer slope of the MUSCL scheme.
#pragma once

#include <math.h>

#include "dvm_internal.cuh"

namespace dvm {
namespace {

// Primitive variables (Eqs. Mo and E): rho, u, theta.  Written without
// contractions so that the value matches a plain IEEE evaluation bit for bit
// (alpha and the number of Euler sub-steps depend on it).
template <int D>
__device__ inline void primitives(const double* U, double& rho, double u[3], double& theta) {
  rho = U[0];
  double u2 = 0.0;
  u[0] = u[1] = u[2] = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = __ddiv_rn(U[1 + i], rho);
    u2 = __dadd_rn(u2, __dmul_rn(u[i], u[i]));
  }
  theta = __ddiv_rn(__dsub_rn(__ddiv_rn(__dmul_rn(2.0, U[D + 1]), rho), u2), (double)D);
}

// Sums over one velocity axis of g(k) = exp(-(v_k - u)^2 / (2 theta)) times
// 1, v_k, v_k^2, in FP64.  The Gaussian is evaluated from its peak outwards
// with the recurrence g(k+1) = g(k) r_k, r_{k+1} = r_k q, q = exp(-dv^2/theta)
// (ratios of consecutive Gaussian samples on a uniform grid): three
// exponentials per axis instead of one per velocity.
__device__ void gauss_axis_sums(int n, int kmin, double dv, double u, double theta, double& G0,
                                double& G1, double& G2) {
  const double h = 0.5 / theta;
  int k0 = (int)floor(u / dv + 0.5) - kmin;
  k0 = k0 < 0 ? 0 : (k0 >= n ? n - 1 : k0);
  const double v0 = (kmin + k0) * dv;
  const double g0 = exp(-(v0 - u) * (v0 - u) * h);
  const double q = exp(-2.0 * dv * dv * h);
  G0 = g0;
  G1 = v0 * g0;
  G2 = v0 * v0 * g0;
  double g = g0, r = exp(-(2.0 * (v0 - u) * dv + dv * dv) * h);
  for (int k = k0 + 1; k < n; ++k) {
    g *= r;
    r *= q;
    const double v = (kmin + k) * dv;
    G0 += g;
    G1 += v * g;
    G2 += v * v * g;
  }
  g = g0;
  double s = exp((2.0 * (v0 - u) * dv - dv * dv) * h);
  for (int k = k0 - 1; k >= 0; --k) {
    g *= s;
    s *= q;
    const double v = (kmin + k) * dv;
    G0 += g;
    G1 += v * g;
    G2 += v * v * g;
  }
}

// Same sums with FP32 samples exp2(-(v - u)^2 log2(e) / (2 theta)) and FP32
// accumulation, for the FP32-storage builds.
__device__ void gauss_axis_sums_f32(int n, int kmin, float dv, float u, float theta, double& G0,
                                    double& G1, double& G2) {
  const float h2 = 0.72134752044448170f / theta;  // log2(e) / 2
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int k = 0; k < n; ++k) {
    const float v = (kmin + k) * dv;
    const float dd = v - u;
    const float gk = exp2f(-h2 * dd * dd);
    s0 += gk;
    s1 = fmaf(v, gk, s1);
    s2 = fmaf(v * v, gk, s2);
  }
  G0 = s0;
  G1 = s1;
  G2 = s2;
}

// Euler flux along dir (Eq. sys1), gamma = 1 + 2/d; zero density carries no
// flux (only reached for lambda = 1, where W = 0).
// Division in the Euler solver: IEEE in the FP64 build, the fast
// approximate quotient (two ulp) in the FP32-storage builds.
__device__ inline double e_div(double a, double b) { return a / b; }
__device__ inline float e_div(float a, float b) { return __fdividef(a, b); }

template <typename TF, int D>
__device__ inline void euler_flux(const TF* U, int dir, TF* F) {
  const TF rho = U[0];
  TF u[3] = {TF(0), TF(0), TF(0)}, ke = TF(0);
  if (rho != TF(0)) {
    const TF ir = e_div(TF(1), rho);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      u[j] = U[1 + j] * ir;
      ke += TF(0.5) * U[1 + j] * u[j];
    }
  }
  const TF pr = (TF(2) / TF(D)) * (U[D + 1] - ke);
  F[0] = U[1 + dir];
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = U[1 + j] * u[dir] + (j == dir ? pr : TF(0));
  F[D + 1] = (U[D + 1] + pr) * u[dir];
}

// van Leer limited slope b phi(a / b), phi(chi) = (|chi| + chi) / (1 + chi),
// in product form (zero unless a b > 0).
template <typename TF, bool LIMITED>
__device__ inline TF slope(TF a, TF b) {
  if (!LIMITED) return b;
  const TF ab = a * b;
  return ab > TF(0) ? e_div(ab + ab, a + b) : TF(0);
}

// Grid-wide barrier of the cooperative Euler launch on a 64-bit arrival
// counter that only grows: a block takes a ticket and waits until the count
// reaches the end of its ticket's generation, ceil((ticket + 1) / n) n with n
// the blocks of the launch (every launch of a handle completes whole
// generations, so the count is a multiple of n between launches).  No block
// resets or republishes anything, so the last arrival releases the others
// with its own atomic.  The wait is bounded (2^31 SM clock cycles, about a
// second); on timeout the status word gets DVM_ERR_TIMEOUT and false is
// returned so that the kernel can leave.
__device__ inline unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_sync(unsigned long long* bar, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long n = gridDim.x;
    __threadfence();
    const unsigned long long ticket = atomicAdd(bar, 1ull);
    const unsigned long long target = (ticket / n + 1) * n;
    int good = 1;
    if (ticket + 1 != target) {
      const long long t0 = clock64();
      while (ld_acquire_u64(bar) < target) {
        if (clock64() - t0 > (1LL << 31)) {
          set_status(status, DVM_ERR_TIMEOUT);
          good = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// alpha_i contribution of one cell: |u_i| + sqrt(gamma theta), gamma = 1 + 2/d
// (largest eigenvalue of the Euler system along i), evaluated without
// contractions like the primitive variables.
template <int D>
__device__ inline void alpha_of(const double* Uc, double a[3]) {
  double rho, u[3], theta;
  primitives<D>(Uc, rho, u, theta);
  const double gamma = __dadd_rn(1.0, __ddiv_rn(2.0, (double)D));
  const double cs = sqrt(__dmul_rn(gamma, theta));
  a[0] = a[1] = a[2] = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) a[i] = (rho > 0.0 && theta > 0.0) ? __dadd_rn(fabs(u[i]), cs) : 0.0;
}

// alpha contribution of one Euler state W (per direction |u_i| + sqrt(gamma
// theta)); zero density (lambda = 1 makes W = 0) carries no wave.  FP64 states
// are evaluated without contractions (same values as a plain IEEE
// evaluation), FP32 states in FP32.
template <int D>
__device__ inline void state_alpha_of(const double* W, double a[3]) {
  a[0] = a[1] = a[2] = 0.0;
  if (W[0] == 0.0) return;
  alpha_of<D>(W, a);
}
template <int D>
__device__ inline void state_alpha_of(const float* W, float a[3]) {
  a[0] = a[1] = a[2] = 0.f;
  if (W[0] == 0.f) return;
  const float ir = __fdividef(1.f, W[0]);
  float u2 = 0.f, u[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = W[1 + i] * ir;
    u2 = fmaf(u[i], u[i], u2);
  }
  const float theta = (2.f * W[D + 1] * ir - u2) * (1.f / D);
  const float cs = sqrtf(fmaxf((1.f + 2.f / D) * theta, 0.f));
#pragma unroll
  for (int i = 0; i < D; ++i) a[i] = fabsf(u[i]) + cs;
}
template <int D>
__device__ inline void state_alpha_of(const float* W, double a[3]) {
  float af[3];
  state_alpha_of<D>(W, af);
  for (int i = 0; i < 3; ++i) a[i] = (double)af[i];
}

template <int D>
__device__ inline void cell_coords(const Geom& g, long long c, int x[3]) {
  x[0] = (int)(c % g.nx[0]);
  x[1] = D > 1 ? (int)((c / g.nx[0]) % g.nx[1]) : 0;
  x[2] = D > 2 ? (int)(c / ((long long)g.nx[0] * g.nx[1])) : 0;
}

__device__ inline long long cell_index(const Geom& g, const int x[3]) {
  return x[0] + (long long)g.nx[0] * (x[1] + (long long)g.nx[1] * x[2]);
}

// mu = (C C^T)^{-1} (U - C M[U]) of Eq. minimMax, with C M[U] from the
// separable factors of the Maxwellian.  Returns 0 or an error code.
template <int D>
__device__ int cell_mu(const Geom& g, const double* A, const double* Uc, double mu[kMaxM],
                       double& rho, double u[3], double& theta) {
  constexpr int NM = D + 2;
#pragma unroll
  for (int i = 0; i < NM; ++i)
    if (!isfinite(Uc[i])) return DVM_ERR_NONFINITE;
  primitives<D>(Uc, rho, u, theta);
  if (!(rho > 0.0) || !(theta > 0.0)) return DVM_ERR_NONPHYSICAL;
  double G0[3], G1[3], G2[3];
#pragma unroll
  for (int i = 0; i < D; ++i) gauss_axis_sums(g.nv[i], g.kmin[i], g.dv, u[i], theta, G0[i], G1[i], G2[i]);
  const double pref = g.w * rho * pow(2.0 * M_PI * theta, -0.5 * D);
  double CM[kMaxM];
  double all = 1.0;
#pragma unroll
  for (int i = 0; i < D; ++i) all *= G0[i];
  CM[0] = pref * all;
  double e = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double other = 1.0;
#pragma unroll
    for (int i = 0; i < D; ++i)
      if (i != j) other *= G0[i];
    CM[1 + j] = pref * G1[j] * other;
    e += G2[j] * other;
  }
  CM[D + 1] = 0.5 * pref * e;
  double r[kMaxM];
#pragma unroll
  for (int i = 0; i < NM; ++i) r[i] = Uc[i] - CM[i];
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < NM; ++j) s += A[i * NM + j] * r[j];
    mu[i] = s;
  }
  return 0;
}

// FP32-storage builds: the same mu with the primitives, the Gaussian sums
// and C M[U] in FP32 (the accuracy of the FP32 Maxwellian samples the kinetic
// pass draws from these parameters) and only U - C M[U], the difference of
// two nearly equal moment vectors, in FP64; Af is (C C^T)^{-1} in FP32.
// GB300's FP64 rate is about 1/64 of its FP32 rate and the end-of-step kernel
// is bound by it otherwise.  A theta that rounds to <= 0 in FP32 is
// recomputed in FP64 before the cell is declared non-physical.
template <int D>
__device__ int cell_mu_f32(const Geom& g, const float* Af, const double* Uc, float mu[kMaxM],
                           float& rho, float u[3], float& theta) {
  constexpr int NM = D + 2;
#pragma unroll
  for (int i = 0; i < NM; ++i)
    if (!isfinite(Uc[i])) return DVM_ERR_NONFINITE;
  if (!(Uc[0] > 0.0)) return DVM_ERR_NONPHYSICAL;
  rho = (float)Uc[0];
  const float ir = 1.f / rho;
  float u2 = 0.f;
  u[0] = u[1] = u[2] = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = (float)Uc[1 + i] * ir;
    u2 = fmaf(u[i], u[i], u2);
  }
  theta = (2.f * (float)Uc[D + 1] * ir - u2) * (1.f / D);
  if (!(theta > 0.f) || !(rho > 0.f)) {
    double rd, ud[3], td;
    primitives<D>(Uc, rd, ud, td);
    if (!(rd > 0.0) || !(td > 0.0)) return DVM_ERR_NONPHYSICAL;
    rho = (float)rd;
    theta = (float)td;
    for (int i = 0; i < 3; ++i) u[i] = (float)ud[i];
    if (!(theta > 0.f) || !(rho > 0.f)) return DVM_ERR_NONPHYSICAL;
  }
  // C M[U] in FP64 from the FP32 Gaussian sums: any rounding of it would
  // enter E[U]'s moments (through mu) and accumulate step by step
  double G0[3], G1[3], G2[3];
#pragma unroll
  for (int i = 0; i < D; ++i) gauss_axis_sums_f32(g.nv[i], g.kmin[i], (float)g.dv, u[i], theta, G0[i], G1[i], G2[i]);
  const double pref = g.w * (double)rho * (double)powf(6.283185307179586f * theta, -0.5f * D);
  double CM[kMaxM];
  double all = 1.0;
#pragma unroll
  for (int i = 0; i < D; ++i) all *= G0[i];
  CM[0] = pref * all;
  double e = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double other = 1.0;
#pragma unroll
    for (int i = 0; i < D; ++i)
      if (i != j) other *= G0[i];
    CM[1 + j] = pref * G1[j] * other;
    e += G2[j] * other;
  }
  CM[D + 1] = 0.5 * pref * e;
  float r[kMaxM];
#pragma unroll
  for (int i = 0; i < NM; ++i) r[i] = (float)(Uc[i] - CM[i]);
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < NM; ++j) s = fmaf(Af[i * NM + j], r[j], s);
    mu[i] = s;
  }
  return 0;
}

}  // namespace
}  // namespace dvm
