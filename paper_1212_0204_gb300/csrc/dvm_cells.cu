// dvm_cells.cu -- per-cell kernels of libdvm: moments and conservative
// Maxwellian parameters, the MUSCL Euler solver, the alpha reduction, the
// end-of-step update, initial data and read-back.  These touch O(N_c) data;
// the O(N_c N_v) work lives in dvm_kinetic.cu.
#include <math.h>

#include <mutex>

#include "dvm_internal.cuh"

namespace dvm {
namespace {

constexpr int kBlock = 256;

inline unsigned blocks_for(long long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

__device__ inline void cell_coords(const Geom& g, long long c, int x[3]) {
  x[0] = (int)(c % g.nx[0]);
  x[1] = (int)((c / g.nx[0]) % g.nx[1]);
  x[2] = (int)(c / ((long long)g.nx[0] * g.nx[1]));
}

__device__ inline long long cell_index(const Geom& g, const int x[3]) {
  return x[0] + (long long)g.nx[0] * (x[1] + (long long)g.nx[1] * x[2]);
}

// Primitive variables (Eqs. Mo and E): rho, u, theta.  Written without
// contractions so that the value matches a plain IEEE evaluation bit for bit
// (alpha and the number of Euler sub-steps depend on it).
__device__ inline void primitives(int d, const double* U, double& rho, double u[3],
                                  double& theta) {
  rho = U[0];
  double u2 = 0.0;
  for (int i = 0; i < 3; ++i) u[i] = 0.0;
  for (int i = 0; i < d; ++i) {
    u[i] = __ddiv_rn(U[1 + i], rho);
    u2 = __dadd_rn(u2, __dmul_rn(u[i], u[i]));
  }
  theta = __ddiv_rn(__dsub_rn(__ddiv_rn(__dmul_rn(2.0, U[d + 1]), rho), u2), (double)d);
}

// Sums over one velocity axis of g(k) = exp(-(v_k - u)^2 / (2 theta)) times
// 1, v_k, v_k^2.  The Gaussian is evaluated from its peak outwards with the
// two-term recurrence g(k+1) = g(k) r_k, r_{k+1} = r_k q, q = exp(-dv^2/theta)
// (ratios of consecutive Gaussian samples on a uniform grid), so that one axis
// costs three exponentials.
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

// mu = (C C^T)^{-1} (U - C M[U]) of Eq. minimMax, with C M[U] from the
// separable factors of the Maxwellian.  Returns 0 or an error code.
__device__ int cell_mu(const Geom& g, const double* A, const double* Uc, double mu[kMaxM],
                       double& rho, double u[3], double& theta) {
  const int d = g.d, nm = g.nm;
  for (int i = 0; i < nm; ++i)
    if (!isfinite(Uc[i])) return DVM_ERR_NONFINITE;
  primitives(d, Uc, rho, u, theta);
  if (!(rho > 0.0) || !(theta > 0.0)) return DVM_ERR_NONPHYSICAL;
  double G0[3], G1[3], G2[3];
  for (int i = 0; i < d; ++i) gauss_axis_sums(g.nv[i], g.kmin[i], g.dv, u[i], theta, G0[i], G1[i], G2[i]);
  const double pref = g.w * rho * pow(2.0 * M_PI * theta, -0.5 * d);
  double CM[kMaxM];
  double all = 1.0;
  for (int i = 0; i < d; ++i) all *= G0[i];
  CM[0] = pref * all;
  double e = 0.0;
  for (int j = 0; j < d; ++j) {
    double other = 1.0;
    for (int i = 0; i < d; ++i)
      if (i != j) other *= G0[i];
    CM[1 + j] = pref * G1[j] * other;
    e += G2[j] * other;
  }
  CM[d + 1] = 0.5 * pref * e;
  double r[kMaxM];
  for (int i = 0; i < nm; ++i) r[i] = Uc[i] - CM[i];
  for (int i = 0; i < nm; ++i) {
    double s = 0.0;
    for (int j = 0; j < nm; ++j) s += A[i * nm + j] * r[j];
    mu[i] = s;
  }
  return 0;
}

// Kinetic-pass parameters of one cell (row layout in dvm_internal.cuh).
template <typename TC>
__device__ void write_params(const Geom& g, TC* prm, long long c, double lam, double weight,
                             double rho, const double u[3], double theta, const double* nu,
                             const double* mu) {
  const int d = g.d, nm = g.nm;
  const long long nc = g.nc;
  const double L = log2(weight) + log2(rho) - 0.5 * d * log2(2.0 * M_PI * theta);
  prm[row_lam() * nc + c] = (TC)lam;
  prm[row_L() * nc + c] = (TC)L;
  for (int i = 0; i < d; ++i) prm[row_u(i) * nc + c] = (TC)u[i];
  prm[row_h(d) * nc + c] = (TC)(M_LOG2E * 0.5 / theta);
  for (int i = 0; i < nm; ++i) {
    prm[row_nu(d, i) * nc + c] = (TC)(nu ? g.w * nu[i] : 0.0);
    prm[row_mu(d, i) * nc + c] = (TC)(weight * g.w * mu[i]);
  }
}

template <typename TC>
__global__ void k_cell_params(Geom g, DevPtrs p, int mode, int initial) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  double Uc[kMaxM], mu[kMaxM], rho, u[3], theta;
  for (int i = 0; i < g.nm; ++i) Uc[i] = p.U[i * g.nc + c];
  const int rc = cell_mu(g, p.A, Uc, mu, rho, u, theta);
  if (rc) {
    set_status(p.status, rc);
    return;
  }
  const double lam = p.lam[c];
  if (mode == 0) {  // E[U] itself, in FP64, to build f^0
    write_params(g, p.eqp, c, lam, 1.0, rho, u, theta, nullptr, mu);
    return;
  }
  // FKS: f^0 carries no deferred equilibrium yet
  const double weight = (g.scheme == DVM_FKS && initial) ? 0.0 : 1.0 - lam;
  write_params(g, (TC*)p.prm, c, lam, weight, rho, u, theta, nullptr, mu);
}

// f^0 = E[U^0] at every phase-space point, from the FP64 equilibrium
// parameters of every cell.
template <typename TS, typename TC>
__global__ void k_init_f(Geom g, DevPtrs p) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nc * g.nvel) return;
  const long long c = idx % g.nc, k = idx / g.nc;
  const int d = g.d;
  const double* prm = p.eqp;
  const long long nc = g.nc;
  int kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
               (int)(k / ((long long)g.nv[0] * g.nv[1]))};
  double q = 0.0, vv = 0.0, lin = (double)prm[row_mu(d, 0) * nc + c];
  for (int i = 0; i < d; ++i) {
    const double v = (double)(g.kmin[i] + kk[i]) * g.dv;
    const double du = v - (double)prm[row_u(i) * nc + c];
    q += du * du;
    vv += v * v;
    lin += (double)prm[row_mu(d, 1 + i) * nc + c] * v;
  }
  lin += (double)prm[row_mu(d, d + 1) * nc + c] * 0.5 * vv;
  const double f = exp2((double)prm[row_L() * nc + c] - (double)prm[row_h(d) * nc + c] * q) + lin;
  StoreT<TS>::store((TS*)p.F + k * nc + c, (TC)f);
}

__global__ void k_prim_to_cons(Geom g, const double* rho, const double* u, const double* T,
                               double* U) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  const int d = g.d;
  const double r = rho[c];
  double ke = 0.0;
  U[c] = r;
  for (int i = 0; i < d; ++i) {
    const double ui = u[i * g.nc + c];
    U[(1 + i) * g.nc + c] = r * ui;
    ke += ui * ui;
  }
  U[(d + 1) * g.nc + c] = 0.5 * r * ke + 0.5 * d * r * T[c];
}

// alpha_i = max_c |u_i| + sqrt(gamma theta) (the largest eigenvalue of the
// Euler system along i, one value per step), W = (1 - lambda) U, and in the
// last block the number of Euler sub-steps from Eq. Time2.
__global__ void __launch_bounds__(kBlock) k_alpha(Geom g, DevPtrs p) {
  __shared__ double red[3][kBlock / 32];
  __shared__ bool last;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int d = g.d, nm = g.nm;
  double a[3] = {0.0, 0.0, 0.0};
  if (c < g.nc) {
    double Uc[kMaxM], rho, u[3], theta;
    for (int i = 0; i < nm; ++i) Uc[i] = p.U[i * g.nc + c];
    primitives(d, Uc, rho, u, theta);
    const double gamma = __dadd_rn(1.0, __ddiv_rn(2.0, (double)d));
    const double cs = sqrt(__dmul_rn(gamma, theta));
    for (int i = 0; i < d; ++i) a[i] = (rho > 0.0 && theta > 0.0) ? __dadd_rn(fabs(u[i]), cs) : 0.0;
    const double w = 1.0 - p.lam[c];
    for (int i = 0; i < nm; ++i) p.W0[i * g.nc + c] = w * Uc[i];
  }
  for (int i = 0; i < 3; ++i) {
    double v = a[i];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) v = fmax(v, red[threadIdx.x][w]);
    atomicMax(&p.alpha_bits[threadIdx.x], (unsigned long long)__double_as_longlong(v));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(p.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double asum = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double ai = __longlong_as_double((long long)atomicExch(&p.alpha_bits[i], 0ull));
    p.alpha[i] = ai;
    if (i < d) asum = __dadd_rn(asum, ai);
  }
  int m;
  if (g.forced_sub > 0) {
    m = g.forced_sub;
  } else {
    const double dtE = __ddiv_rn(__dmul_rn(0.5, g.dx), asum);
    const double r = ceil(__ddiv_rn(g.dt, dtE));
    m = (r < 1.0) ? 1 : (r > 1e9 ? 1000000000 : (int)r);
  }
  if (m > g.m_cap) {
    set_status(p.status, DVM_ERR_CFL);
    m = g.m_cap;
  }
  *p.msub = m;
  *p.counter = 0u;
}

// Euler flux along dir (Eq. sys1), gamma = 1 + 2/d; zero density carries no
// flux (only reached for lambda = 1, where W = 0).
template <typename TF>
__device__ inline void euler_flux(int d, const TF* U, int dir, TF* F) {
  const TF rho = U[0];
  TF u[3] = {TF(0), TF(0), TF(0)}, ke = TF(0);
  if (rho != TF(0)) {
    for (int j = 0; j < d; ++j) {
      u[j] = U[1 + j] / rho;
      ke += TF(0.5) * U[1 + j] * u[j];
    }
  }
  const TF pr = (TF(2) / TF(d)) * (U[d + 1] - ke);
  F[0] = U[1 + dir];
  for (int j = 0; j < d; ++j) F[1 + j] = U[1 + j] * u[dir] + (j == dir ? pr : TF(0));
  F[d + 1] = (U[d + 1] + pr) * u[dir];
}

// van Leer limited slope b phi(a / b), phi(chi) = (|chi| + chi) / (1 + chi),
// in product form (zero unless a b > 0).
template <typename TF, bool LIMITED>
__device__ inline TF slope(TF a, TF b) {
  if (!LIMITED) return b;
  const TF ab = a * b;
  return ab > TF(0) ? (ab + ab) / (a + b) : TF(0);
}

// One forward-Euler MUSCL sub-step (Eq. discmom), unsplit over directions.
// Face fluxes are evaluated in TF; the state stays FP64.
template <typename TF, bool LIMITED>
__global__ void __launch_bounds__(kBlock) k_muscl(Geom g, DevPtrs p, int substep) {
  const int m = *p.msub;
  if (substep >= m) return;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  const int d = g.d, nm = g.nm;
  const double* src = (substep & 1) ? p.W1 : p.W0;
  double* dst = (substep & 1) ? p.W0 : p.W1;
  int x[3];
  cell_coords(g, c, x);
  double acc[kMaxM] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int dir = 0; dir < d; ++dir) {
    TF Us[5][kMaxM], Fs[5][kMaxM];
    for (int o = -2; o <= 2; ++o) {
      int y[3] = {x[0], x[1], x[2]};
      const int n = g.nx[dir];
      if (g.bc[dir] == DVM_BC_PERIODIC) {
        y[dir] = wrap((long long)x[dir] + o, n);
      } else {
        const int t = x[dir] + o;
        y[dir] = t < 0 ? 0 : (t >= n ? n - 1 : t);
      }
      const long long cc = cell_index(g, y);
      for (int i = 0; i < nm; ++i) Us[o + 2][i] = (TF)src[i * g.nc + cc];
      euler_flux<TF>(d, Us[o + 2], dir, Fs[o + 2]);
    }
    const TF al = (TF)p.alpha[dir];
    for (int i = 0; i < nm; ++i) {
      TF Gp[5], Gm[5];
      for (int s = 0; s < 5; ++s) {
        Gp[s] = Fs[s][i] + al * Us[s][i];
        Gm[s] = Fs[s][i] - al * Us[s][i];
      }
      // face j+1/2 between cells (1, 2) and (2, 3) of the 5-cell stencil
      TF psi[2];
      for (int f = 0; f < 2; ++f) {
        const int j = 1 + f;
        const TF sp = slope<TF, LIMITED>(Gp[j] - Gp[j - 1], Gp[j + 1] - Gp[j]);
        const TF sm = slope<TF, LIMITED>(Gm[j + 1] - Gm[j], Gm[j + 2] - Gm[j + 1]);
        psi[f] = TF(0.5) * (Fs[j][i] + Fs[j + 1][i]) - TF(0.5) * al * (Us[j + 1][i] - Us[j][i]) +
                 TF(0.25) * (sp - sm);
      }
      acc[i] += (double)psi[1] - (double)psi[0];
    }
  }
  const double k = (g.dt / m) / g.dx;
  for (int i = 0; i < nm; ++i) dst[i * g.nc + c] = src[i * g.nc + c] - k * acc[i];
}

// Outflow: snapshot of the boundary pieces of every velocity before the
// in-place kinetic pass overwrites them (1D: cells 0 and N-1).
template <typename TS>
__global__ void k_ghost1d(Geom g, DevPtrs p) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= g.nvel) return;
  const long long n = *p.step;
  const long long o = transport_offset(g.kmin[0] + k, n, g.p);
  const int N = g.nx[0];
  const TS* F = (const TS*)p.F + k * g.nc;
  TS* G = (TS*)p.ghost;
  G[2 * k] = F[wrap(0 - o, N)];
  G[2 * k + 1] = F[wrap((long long)(N - 1) - o, N)];
}

// End of a step: U^{n+1}, the HOFKS correction nu = A (U_E - U_M)
// (Eq. minim_full), checks, and the parameters of the next pass.
template <typename TC, int SCHEME>
__global__ void k_finalize(Geom g, DevPtrs p) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c == 0) *p.step += 1;
  if (c >= g.nc) return;
  const int nm = g.nm;
  const long long nc = g.nc;
  double Un[kMaxM], nu[kMaxM];
  const bool hofks = SCHEME != DVM_FKS;
  const int nacc = hofks ? 2 * nm : nm;
  double sums[2 * kMaxM];
  for (int j = 0; j < nacc; ++j) {
    double s = 0.0;
    for (int sp = 0; sp < g.nsplit; ++sp) s += p.acc[((long long)sp * 2 * nm + j) * nc + c];
    sums[j] = g.w * s;
  }
  if (hofks) {
    const double* UE = (*p.msub & 1) ? p.W1 : p.W0;
    double r[kMaxM];
    for (int i = 0; i < nm; ++i) {
      const double ue = UE[i * nc + c];
      r[i] = ue - sums[nm + i];
      Un[i] = sums[i] + ue;
      p.Us[i * nc + c] = sums[i];
      p.UM[i * nc + c] = sums[nm + i];
    }
    for (int i = 0; i < nm; ++i) {
      double s = 0.0;
      for (int j = 0; j < nm; ++j) s += p.A[i * nm + j] * r[j];
      nu[i] = s;
    }
  } else {
    for (int i = 0; i < nm; ++i) {
      Un[i] = sums[i];
      p.Us[i * nc + c] = sums[i];
    }
  }
  for (int i = 0; i < nm; ++i) p.U[i * nc + c] = Un[i];
  double mu[kMaxM], rho, u[3], theta;
  const int rc = cell_mu(g, p.A, Un, mu, rho, u, theta);
  if (rc) {
    set_status(p.status, rc);
    return;
  }
  const double lam = p.lam[c];
  write_params(g, (TC*)p.prm, c, lam, 1.0 - lam, rho, u, theta, hofks ? nu : nullptr, mu);
}

// f at the cell centres: stored piece value plus the deferred term.
template <typename TS, typename TC>
__global__ void k_materialize(Geom g, DevPtrs p, double* out) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nc * g.nvel) return;
  const long long c = idx % g.nc, k = idx / g.nc;
  const int d = g.d;
  const long long n = *p.step, nc = g.nc;
  const TC* prm = (const TC*)p.prm;
  int x[3], kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
                     (int)(k / ((long long)g.nv[0] * g.nv[1]))};
  cell_coords(g, c, x);
  int q[3] = {0, 0, 0};
  double v[3] = {0.0, 0.0, 0.0}, vv = 0.0;
  for (int i = 0; i < d; ++i) {
    const long long kg = g.kmin[i] + kk[i];
    q[i] = wrap((long long)x[i] - transport_offset(kg, n, g.p), g.nx[i]);
    v[i] = (double)kg * g.dv;
    vv += v[i] * v[i];
  }
  vv *= 0.5;
  const long long slot = cell_index(g, q);
  double f = (double)StoreT<TS>::load((const TS*)p.F + k * nc + slot);
  if (g.scheme == DVM_FKS) {
    double qq = 0.0, lin = (double)prm[row_mu(d, 0) * nc + c];
    for (int i = 0; i < d; ++i) {
      const double du = v[i] - (double)prm[row_u(i) * nc + c];
      qq += du * du;
      lin += (double)prm[row_mu(d, 1 + i) * nc + c] * v[i];
    }
    lin += (double)prm[row_mu(d, d + 1) * nc + c] * vv;
    f += exp2((double)prm[row_L() * nc + c] - (double)prm[row_h(d) * nc + c] * qq) + lin;
  } else {
    double lin = (double)prm[row_nu(d, 0) * nc + c];
    for (int i = 0; i < d; ++i) lin += (double)prm[row_nu(d, 1 + i) * nc + c] * v[i];
    lin += (double)prm[row_nu(d, d + 1) * nc + c] * vv;
    f += lin;
  }
  out[k * nc + c] = f;
}

__global__ void k_offsets(Geom g, long long n, long long* out, int width) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / width, k = t % width;
  if (i >= g.d || k >= g.nv[i]) return;
  out[i * width + k] = transport_offset(g.kmin[i] + k, n, g.p);
}

}  // namespace

// ------------------------------------------------------------ launchers

void launch_prim_to_cons(const Geom& g, const double* rho, const double* u, const double* T,
                         double* U, cudaStream_t s) {
  k_prim_to_cons<<<blocks_for(g.nc), kBlock, 0, s>>>(g, rho, u, T, U);
}

void launch_cell_params(const Geom& g, const DevPtrs& p, int mode, int initial, cudaStream_t s) {
  if (g.precision == DVM_F64)
    k_cell_params<double><<<blocks_for(g.nc), kBlock, 0, s>>>(g, p, mode, initial);
  else
    k_cell_params<float><<<blocks_for(g.nc), kBlock, 0, s>>>(g, p, mode, initial);
}

void launch_init_f(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  const unsigned nb = blocks_for(g.nc * g.nvel);
  if (g.precision == DVM_F64)
    k_init_f<double, double><<<nb, kBlock, 0, s>>>(g, p);
  else if (g.precision == DVM_F32)
    k_init_f<float, float><<<nb, kBlock, 0, s>>>(g, p);
  else
    k_init_f<__nv_bfloat16, float><<<nb, kBlock, 0, s>>>(g, p);
}

void launch_alpha(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  k_alpha<<<blocks_for(g.nc), kBlock, 0, s>>>(g, p);
}

void launch_muscl(const Geom& g, const DevPtrs& p, int substep, cudaStream_t s) {
  const bool lim = g.scheme == DVM_HOFKS;
  const unsigned nb = blocks_for(g.nc);
  if (g.precision == DVM_F64) {
    if (lim) k_muscl<double, true><<<nb, kBlock, 0, s>>>(g, p, substep);
    else k_muscl<double, false><<<nb, kBlock, 0, s>>>(g, p, substep);
  } else {
    if (lim) k_muscl<float, true><<<nb, kBlock, 0, s>>>(g, p, substep);
    else k_muscl<float, false><<<nb, kBlock, 0, s>>>(g, p, substep);
  }
}

void launch_ghost(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  if (g.ghost_mode == 1) {
    const unsigned nb = blocks_for(g.nvel);
    if (g.precision == DVM_F64) k_ghost1d<double><<<nb, kBlock, 0, s>>>(g, p);
    else if (g.precision == DVM_F32) k_ghost1d<float><<<nb, kBlock, 0, s>>>(g, p);
    else k_ghost1d<__nv_bfloat16><<<nb, kBlock, 0, s>>>(g, p);
  } else if (g.ghost_mode == 2) {
    const size_t es = g.precision == DVM_F64 ? 8 : (g.precision == DVM_F32 ? 4 : 2);
    cudaMemcpyAsync(p.ghost, p.F, es * (size_t)g.nc * (size_t)g.nvel, cudaMemcpyDeviceToDevice, s);
  }
}

void launch_finalize(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  const unsigned nb = blocks_for(g.nc);
  const bool f64 = g.precision == DVM_F64;
  if (g.scheme == DVM_FKS) {
    if (f64) k_finalize<double, DVM_FKS><<<nb, kBlock, 0, s>>>(g, p);
    else k_finalize<float, DVM_FKS><<<nb, kBlock, 0, s>>>(g, p);
  } else {
    if (f64) k_finalize<double, DVM_HOFKS><<<nb, kBlock, 0, s>>>(g, p);
    else k_finalize<float, DVM_HOFKS><<<nb, kBlock, 0, s>>>(g, p);
  }
}

void launch_materialize(const Geom& g, const DevPtrs& p, double* out, cudaStream_t s) {
  const unsigned nb = blocks_for(g.nc * g.nvel);
  if (g.precision == DVM_F64)
    k_materialize<double, double><<<nb, kBlock, 0, s>>>(g, p, out);
  else if (g.precision == DVM_F32)
    k_materialize<float, float><<<nb, kBlock, 0, s>>>(g, p, out);
  else
    k_materialize<__nv_bfloat16, float><<<nb, kBlock, 0, s>>>(g, p, out);
}

void launch_offsets(const Geom& g, long long n, long long* out, int width, cudaStream_t s) {
  k_offsets<<<blocks_for(3LL * width, 128), 128, 0, s>>>(g, n, out, width);
}

}  // namespace dvm

// ---------------------------------------------------------------------------
// Allocation-free equilibrium (dvm_equilibrium_noalloc in dvm.h).
//
// For callers that may not allocate device memory (code inside a fixed
// memory budget, or a host thread that must not call into the allocator):
// the per-cell scratch of the f^0 = E[U] initialisation -- the status word,
// (C C^T)^{-1} and the FP64 equilibrium parameters of every cell -- lives in
// this file-scope device array instead of a workspace.  Every GPU that loads
// the library holds it until the process exits.  Host code must not use the
// symbol itself as a device address: its device address is looked up once
// per device with cudaGetSymbolAddress.
namespace dvm {
namespace {

constexpr size_t kNoAllocBytes = DVM_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[256] = {};

// Device address of the scratch array on the current device (looked up on the
// first call per device).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dvm

extern "C" int dvm_equilibrium_noalloc(const dvm_config* cfg, const double* U, double* f,
                                       void* cuda_stream) {
  using namespace dvm;
  Geom g;
  std::string msg;
  if (make_geom(cfg, &g, &msg) != 0 || !U || !f) return DVM_ERR_ARG;
  g.precision = DVM_F64;  // FP64 output, FP64 parameters
  // scratch layout: [0, 256) status word and (C C^T)^{-1}; then the
  // equilibrium parameters (prm_rows x Nc); then Nc doubles read as lambda
  const size_t nc = (size_t)g.nc;
  const size_t need = 256 + 8 * (size_t)prm_rows(g.d) * nc + 8 * nc;
  if (need > kNoAllocBytes) return DVM_ERR_TOO_LARGE;
  double A[kMaxM * kMaxM];
  if (invert_moment_matrix(g, A) != 0) return DVM_ERR_ARG;
  void* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return DVM_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DevPtrs p;
  memset(&p, 0, sizeof p);
  char* b = (char*)base;
  p.status = (int*)b;
  p.A = (double*)(b + 64);
  p.eqp = (double*)(b + 256);
  p.lam = p.eqp + (size_t)prm_rows(g.d) * nc;
  p.U = const_cast<double*>(U);
  p.F = f;
  // the status word must start at zero; everything else is written before it
  // is read within this call
  if (cudaMemsetAsync(p.status, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(p.A, A, sizeof(double) * g.nm * g.nm, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(p.lam, 0, 8 * nc, s) != cudaSuccess)
    return DVM_ERR_CUDA;
  launch_cell_params(g, p, 0, 1, s);
  launch_init_f(g, p, s);
  int status = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&status, p.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DVM_ERR_CUDA;
  return status;
}
