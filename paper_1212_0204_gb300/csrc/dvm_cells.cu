// dvm_cells.cu -- per-cell kernels of libdvm: moments and conservative
// Maxwellian parameters, the MUSCL Euler solver, the alpha reduction, the
// end-of-step update, initial data and read-back.  These touch O(N_c) data;
// the O(N_c N_v) work lives in dvm_kinetic.cu.
//
// Precision: the FP64 build does everything in FP64.  In the FP32/BF16
// builds (FP32 f) the per-cell work that feeds f is done in FP32 where FP64
// buys nothing beyond f's own rounding -- Maxwellian samples, the Euler
// fluxes and state, logarithms -- and in FP64 where moments are combined:
// partial sums, U^{n+1} = U_* + U_E, U - C M[U], nu and mu.  GB300's FP64
// rate is about 1/60 of its FP32 rate, so this split matters.
#include <math.h>

#include <mutex>
#include <type_traits>

#include "dvm_internal.cuh"
#include "dvm_math.cuh"

namespace dvm {
namespace {

constexpr int kBlock = 256;

inline unsigned blocks_for(long long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

// Kinetic-pass parameters of one cell (row layout in dvm_internal.cuh).
template <typename TC, int D>
__device__ void write_params(const Geom& g, TC* prm, long long c, double lam, double weight,
                             double rho, const double u[3], double theta, const double* nu,
                             const double* mu) {
  constexpr int NM = D + 2;
  const long long nc = g.nc;
  TC L, h;
  if (sizeof(TC) == 8) {
    L = (TC)(log2(weight) + log2(rho) - 0.5 * D * log2(2.0 * M_PI * theta));
    h = (TC)(M_LOG2E * 0.5 / theta);
  } else {
    L = (TC)(log2f((float)weight) + log2f((float)rho) - 0.5f * D * log2f(6.283185307179586f * (float)theta));
    h = (TC)(0.72134752044448170f / (float)theta);
  }
  prm[prm_at(row_lam(), c, nc)] = (TC)lam;
  prm[prm_at(row_L(), c, nc)] = L;
#pragma unroll
  for (int i = 0; i < D; ++i) prm[prm_at(row_u(i), c, nc)] = (TC)u[i];
  prm[prm_at(row_h(D), c, nc)] = h;
  // the energy row holds the coefficient of |v|^2 (half that of |v|^2 / 2)
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    const double e = i == NM - 1 ? 0.5 : 1.0;
    prm[prm_at(row_nu(D, i), c, nc)] = (TC)(nu ? e * g.w * nu[i] : 0.0);
    prm[prm_at(row_mu(D, i), c, nc)] = (TC)(e * weight * g.w * mu[i]);
  }
}

// The same parameters from FP32 primitives and corrections (FP32-storage
// builds; the values the FP64 version rounds to FP32, up to a few ulp).
template <int D>
__device__ void write_params_f32(const Geom& g, float* prm, long long c, float lam, float weight,
                                 float rho, const float u[3], float theta, const float* nu,
                                 const float* mu) {
  constexpr int NM = D + 2;
  const long long nc = g.nc;
  prm[prm_at(row_lam(), c, nc)] = lam;
  prm[prm_at(row_L(), c, nc)] = log2f(weight) + log2f(rho) - 0.5f * D * log2f(6.283185307179586f * theta);
#pragma unroll
  for (int i = 0; i < D; ++i) prm[prm_at(row_u(i), c, nc)] = u[i];
  prm[prm_at(row_h(D), c, nc)] = 0.72134752044448170f / theta;
  const float w = (float)g.w;
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    const float e = i == NM - 1 ? 0.5f : 1.f;
    prm[prm_at(row_nu(D, i), c, nc)] = nu ? e * w * nu[i] : 0.f;
    prm[prm_at(row_mu(D, i), c, nc)] = e * weight * w * mu[i];
  }
}

// (C C^T)^{-1} in FP32 in shared memory (one copy per block)
template <int D>
__device__ inline void stage_af(const DevPtrs& p, float* sA) {
  if (threadIdx.x < (D + 2) * (D + 2)) sA[threadIdx.x] = (float)p.A[threadIdx.x];
  __syncthreads();
}

template <typename TC, int D>
__global__ void k_cell_params(Geom g, DevPtrs p, int mode, int initial) {
  __shared__ float sA[kMaxM * kMaxM];
  if (sizeof(TC) == 4 && mode != 0) stage_af<D>(p, sA);
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  double Uc[kMaxM], mu[kMaxM], rho, u[3], theta;
#pragma unroll
  for (int i = 0; i < D + 2; ++i) Uc[i] = p.U[i * g.nc + c];
  const double lam = p.lam[c];
  if (mode == 0) {  // E[U] itself, in FP64, to build f^0
    const int rc = cell_mu<D>(g, p.A, Uc, mu, rho, u, theta);
    if (rc) {
      set_status(p.status, rc);
      return;
    }
    write_params<double, D>(g, p.eqp, c, lam, 1.0, rho, u, theta, nullptr, mu);
    return;
  }
  // FKS: f^0 carries no deferred equilibrium yet
  const double weight = (g.scheme == DVM_FKS && initial) ? 0.0 : 1.0 - lam;
  if constexpr (sizeof(TC) == 4) {
    float muf[kMaxM], rf, uf[3], tf;
    const int rc = cell_mu_f32<D>(g, sA, Uc, muf, rf, uf, tf);
    if (rc) {
      set_status(p.status, rc);
      return;
    }
    write_params_f32<D>(g, (float*)p.prm, c, (float)lam, (float)weight, rf, uf, tf, nullptr, muf);
  } else {
    const int rc = cell_mu<D>(g, p.A, Uc, mu, rho, u, theta);
    if (rc) {
      set_status(p.status, rc);
      return;
    }
    write_params<TC, D>(g, (TC*)p.prm, c, lam, weight, rho, u, theta, nullptr, mu);
  }
}

template <typename TS> struct ComputeOf { typedef float type; };
template <> struct ComputeOf<double> { typedef double type; };

// f^0 = E[U^0] at every phase-space point, from the FP64 equilibrium
// parameters of every cell, evaluated in the storage's compute type (FP64
// for FP64 storage, FP32 otherwise).
template <typename TS, int D>
__global__ void k_init_f(Geom g, DevPtrs p) {
  typedef typename ComputeOf<TS>::type TC;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nc * g.nvel) return;
  const long long c = idx % g.nc, k = idx / g.nc;
  const double* prm = p.eqp;
  const long long nc = g.nc;
  const int kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
                     (int)(k / ((long long)g.nv[0] * g.nv[1]))};
  TC q = TC(0), vv = TC(0), lin = (TC)prm[prm_at(row_mu(D, 0), c, nc)];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const TC v = (TC)((double)(g.kmin[i] + kk[i]) * g.dv);
    const TC du = v - (TC)prm[prm_at(row_u(i), c, nc)];
    q += du * du;
    vv += v * v;
    lin += (TC)prm[prm_at(row_mu(D, 1 + i), c, nc)] * v;
  }
  lin += (TC)prm[prm_at(row_mu(D, D + 1), c, nc)] * vv;
  const TC e = (TC)prm[prm_at(row_L(), c, nc)] - (TC)prm[prm_at(row_h(D), c, nc)] * q;
  const TC f = (sizeof(TC) == 8 ? (TC)exp2((double)e) : (TC)exp2f((float)e)) + lin;
  StoreT<TS>::store((TS*)p.F + k * nc + c, f);
}

// f^0 = E[U^0] for FP32/BF16 storage, the same FP32 arithmetic as k_init_f:
// one thread per cell converts the cell's FP64 equilibrium parameters once
// and writes a chunk of velocities (blockIdx.y), consecutive threads writing
// consecutive cells of each velocity row; the velocity components come from
// a shared table.  The write of f (4 or 2 bytes a point) is the bound.
template <typename TS, int D>
__global__ void __launch_bounds__(kBlock) k_init_f_rows(Geom g, DevPtrs p, int kchunk) {
  __shared__ float s_v[kMaxD][kMaxV1];
  for (int t = threadIdx.x; t < D * kMaxV1; t += blockDim.x) {
    const int i = t / kMaxV1, kk = t % kMaxV1;
    if (kk < g.nv[i]) s_v[i][kk] = (float)((double)(g.kmin[i] + kk) * g.dv);
  }
  __syncthreads();
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  const long long nc = g.nc;
  const double* prm = p.eqp;
  float u[3], m[kMaxD];
  const float L = (float)prm[prm_at(row_L(), c, nc)], h = (float)prm[prm_at(row_h(D), c, nc)];
  const float mu0 = (float)prm[prm_at(row_mu(D, 0), c, nc)];
  const float mu4 = (float)prm[prm_at(row_mu(D, D + 1), c, nc)];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = (float)prm[prm_at(row_u(i), c, nc)];
    m[i] = (float)prm[prm_at(row_mu(D, 1 + i), c, nc)];
  }
  const long long kb = (long long)blockIdx.y * kchunk;
  const long long ke = kb + kchunk < g.nvel ? kb + kchunk : g.nvel;
  int kk[3] = {(int)(kb % g.nv[0]), D > 1 ? (int)((kb / g.nv[0]) % g.nv[1]) : 0,
               D > 2 ? (int)(kb / ((long long)g.nv[0] * g.nv[1])) : 0};
  TS* F = (TS*)p.F + c;
  for (long long k = kb; k < ke; ++k) {
    float q = 0.f, vv = 0.f, lin = mu0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float v = s_v[i][kk[i]];
      const float du = v - u[i];
      q += du * du;
      vv += v * v;
      lin += m[i] * v;
    }
    lin += mu4 * vv;
    const float e = L - h * q;
    StoreT<TS>::store(F + k * nc, exp2f(e) + lin);
    if (++kk[0] == g.nv[0]) {
      kk[0] = 0;
      if (D > 1 && ++kk[1] == g.nv[1]) {
        kk[1] = 0;
        if (D > 2) ++kk[2];
      }
    }
  }
}

template <int D>
__global__ void k_prim_to_cons(Geom g, const double* rho, const double* u, const double* T,
                               double* U) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  const double r = rho[c];
  double ke = 0.0;
  U[c] = r;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const double ui = u[i * g.nc + c];
    U[(1 + i) * g.nc + c] = r * ui;
    ke += ui * ui;
  }
  U[(D + 1) * g.nc + c] = 0.5 * r * ke + 0.5 * D * r * T[c];
}

// ------------------------------------------------------------ alpha and m

// Block max of alpha, atomically merged; the last block to finish publishes
// the three maxima as the alpha of the first Euler sub-step (slot 0), clears
// the other two slots and resets the reduction.  FP32 values are reduced in
// FP32: their maximum is one of them, so the published double is the same as
// from a reduction in FP64.
template <int D, typename TA>
__device__ void alpha_reduce_publish(const Geom& g, const DevPtrs& p, const TA a[3]) {
  __shared__ TA red[3][kBlock / 32];
  __shared__ bool last;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    TA v = a[i];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    TA v = 0;
    for (int w = 0; w < kBlock / 32; ++w) v = fmax(v, red[threadIdx.x][w]);
    atomicMax(&p.alpha_bits[threadIdx.x], (unsigned long long)__double_as_longlong((double)v));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(p.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  for (int i = 0; i < 3; ++i) {
    p.aslot[i] = atomicExch(&p.alpha_bits[i], 0ull);
    p.aslot[3 + i] = 0ull;
    p.aslot[6 + i] = 0ull;
  }
  *p.counter = 0u;
}

// alpha, W = (1 - lambda) U and the sub-step count from the current moments
// (used once after a state is set; afterwards the end-of-step kernel does it).
template <typename TW, int D>
__global__ void __launch_bounds__(kBlock) k_alpha(Geom g, DevPtrs p) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double a[3] = {0.0, 0.0, 0.0};
  if (c < g.nc) {
    TW W[kMaxM];
    const double w = 1.0 - p.lam[c];
#pragma unroll
    for (int i = 0; i < D + 2; ++i) {
      W[i] = (TW)(w * p.U[i * g.nc + c]);
      ((TW*)p.W0)[i * g.nc + c] = W[i];
    }
    state_alpha_of<D>(W, a);
  }
  alpha_reduce_publish<D, double>(g, p, a);
}

// ---------------------------------------------------------------- MUSCL

// Tiles of the Euler sub-step: TX x TY cells of one z plane, one thread per
// cell, staged with a two-cell halo in every active direction; the face
// fluxes of the tile (one more face than cells along each direction) are
// kept in shared memory as well.
template <int D, typename TF>
struct ETile {
  static constexpr int TX = D == 1 ? 128 : 32;
  static constexpr int TY = D == 1 ? 1 : 4;
  static constexpr int SX = TX + 4;
  static constexpr int SY = D >= 2 ? TY + 4 : 1;
  static constexpr int SZ = D == 3 ? 5 : 1;
  static constexpr int NS = SX * SY * SZ;   // staged cells
  static constexpr int FX = TX + 1, FY = D >= 2 ? TY + 1 : 1, FZ = D == 3 ? 2 : 1;
  static constexpr int NF = FX * FY * FZ;   // face slots per direction
  static constexpr int CELLS = TX * TY;
  static constexpr int THREADS = CELLS * D;  // one thread per (cell, direction)
  static constexpr size_t SMEM = (size_t)(D + 2) * (NS + D * NF) * sizeof(TF);
};

__device__ inline int bc_index(int t, int n, int bc) {
  if (bc == DVM_BC_PERIODIC) {
    if (t >= 0 && t < n) return t;
    const int r = t % n;  // 32-bit: |t| < n + 3
    return r < 0 ? r + n : r;
  }
  return t < 0 ? 0 : (t >= n ? n - 1 : t);
}

// Numerical flux psi_{j+1/2} of Eq. discmom along dir, component by
// component, from the four staged cells j-1, j, j+1, j+2 (index c of cell j,
// stride st along dir).
template <typename TF, bool LIMITED, int D>
__device__ inline void face_flux(const TF* sw, int ns, int c, int st, int dir, TF al, TF psi[D + 2]) {
  constexpr int NM = D + 2;
  TF Us[4][NM], Fs[4][NM];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
#pragma unroll
    for (int i = 0; i < NM; ++i) Us[o][i] = sw[i * ns + c + (o - 1) * st];
    euler_flux<TF, D>(Us[o], dir, Fs[o]);
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    TF Gp[4], Gm[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      Gp[o] = Fs[o][i] + al * Us[o][i];
      Gm[o] = Fs[o][i] - al * Us[o][i];
    }
    // sigma^+_j from (j-1, j, j+1), sigma^-_{j+1} from (j, j+1, j+2)
    const TF sp = slope<TF, LIMITED>(Gp[1] - Gp[0], Gp[2] - Gp[1]);
    const TF sm = slope<TF, LIMITED>(Gm[2] - Gm[1], Gm[3] - Gm[2]);
    psi[i] = TF(0.5) * (Fs[1][i] + Fs[2][i]) - TF(0.5) * al * (Us[2][i] - Us[1][i]) +
             TF(0.25) * (sp - sm);
  }
}

// Face fluxes of one tile along DIR (compile-time): slot (fx, fy, fz) holds
// the face on the low side of local cell (fx, fy, fz); slot + 1 along DIR is
// the high side.  The thread computes its cell's high face, and the first
// cell along DIR also its low face.
template <typename TF, bool LIMITED, int D, int DIR>
__device__ inline void tile_faces(const TF* sw, TF* sf, int ctr, int tx, int ty, TF al) {
  using T = ETile<D, TF>;
  constexpr int NM = D + 2;
  constexpr int st = DIR == 0 ? 1 : (DIR == 1 ? T::SX : T::SX * T::SY);
  constexpr int fst = DIR == 0 ? 1 : (DIR == 1 ? T::FX : T::FX * T::FY);
  const int fbase = tx + T::FX * ty;
  TF* sfd = sf + DIR * NM * T::NF;
  TF psi[NM];
  face_flux<TF, LIMITED, D>(sw, T::NS, ctr, st, DIR, al, psi);
#pragma unroll
  for (int c = 0; c < NM; ++c) sfd[c * T::NF + fbase + fst] = psi[c];
  const bool first = DIR == 0 ? tx == 0 : (DIR == 1 ? ty == 0 : true);
  if (first) {
    face_flux<TF, LIMITED, D>(sw, T::NS, ctr - st, st, DIR, al, psi);
#pragma unroll
    for (int c = 0; c < NM; ++c) sfd[c * T::NF + fbase] = psi[c];
  }
}

// All m MUSCL sub-steps of one kinetic step (Section 4.3.2, Eq. discmom:
// forward Euler, unsplit over directions) in one cooperative launch:
// W_0 -> W_1 -> ... with a grid barrier between sub-steps; U_E = W_{m mod 2}.
// Per tile and sub-step: stage the tile and its halo in shared memory (loads
// bypass L1: other blocks rewrite the buffers between sub-steps), compute each
// face flux once, then update every cell from its two faces per direction.
// Arithmetic in TF (FP64 in the FP64 build, FP32 in the FP32-storage builds).
template <typename TF, bool LIMITED, int D>
__global__ void __launch_bounds__(ETile<D, TF>::THREADS) k_euler(Geom g, DevPtrs p) {
  using T = ETile<D, TF>;
  constexpr int NM = D + 2;
  extern __shared__ unsigned char s_raw[];
  __shared__ TF s_amax[3][T::THREADS / 32];
  TF* sw = reinterpret_cast<TF*>(s_raw);  // [NM][SZ][SY][SX]
  TF* sf = sw + NM * T::NS;               // [D][NM][FZ][FY][FX]
  const int Nx = g.nx[0], Ny = g.nx[1], Nz = g.nx[2];
  const long long nc = g.nc;
  const int ntx = (Nx + T::TX - 1) / T::TX, nty = (Ny + T::TY - 1) / T::TY;
  const int ntiles = ntx * nty * Nz;
  const int tid = threadIdx.x;
  const int cid = tid % T::CELLS, mydir = tid / T::CELLS;
  const int tx = cid % T::TX, ty = cid / T::TX;
  const int cz = D == 3 ? 2 : 0, cy = D >= 2 ? ty + 2 : 0, cx = tx + 2;
  const int ctr = cx + T::SX * (cy + T::SY * cz);  // staged index of this thread's cell
  // per sub-step scalars, computed in FP64 by thread 0 only and broadcast
  __shared__ double s_dtE;
  __shared__ TF s_k, s_al[3];
  __shared__ int s_last, s_bad;
  double t = 0.0, a0[3] = {0.0, 0.0, 0.0};
  // stage tile `tile` of the state src with its two-cell halo (loads bypass
  // L1: other blocks rewrite the buffers between sub-steps)
  auto stage = [&](const TF* src, int tile) {
    const int x0 = (tile % ntx) * T::TX;
    const int y0 = ((tile / ntx) % nty) * T::TY;
    const int z = tile / (ntx * nty);
    for (int i = tid; i < T::NS; i += T::THREADS) {
      const int lx = i % T::SX, ly = (i / T::SX) % T::SY, lz = i / (T::SX * T::SY);
      const int gx = bc_index(x0 - 2 + lx, Nx, g.bc[0]);
      const int gy = D >= 2 ? bc_index(y0 - 2 + ly, Ny, g.bc[1]) : 0;
      const int gz = D == 3 ? bc_index(z - 2 + lz, Nz, g.bc[2]) : 0;
      const long long cc = gx + (long long)Nx * (gy + (long long)Ny * gz);
#pragma unroll
      for (int c = 0; c < NM; ++c) sw[c * T::NS + i] = __ldcg(src + c * nc + cc);
    }
  };
  int s = 0;
  for (;; ++s) {
    const TF* src = (const TF*)((s & 1) ? p.W1 : p.W0);
    TF* dst = (TF*)((s & 1) ? p.W0 : p.W1);
    // thread 0 issues its reads of the barrier generation and of this
    // sub-step's alpha first; their latency overlaps the first tile's staging
    double ad[3] = {0.0, 0.0, 0.0};
    if (tid == 0) {
      // alpha of this sub-step's initial state: slot s % 3, complete since the
      // barrier that ended the previous sub-step
#pragma unroll
      for (int d = 0; d < 3; ++d) ad[d] = __longlong_as_double((long long)__ldcg(p.aslot + (s % 3) * 3 + d));
    }
    if ((int)blockIdx.x < ntiles) stage(src, blockIdx.x);
    if (tid == 0) {
      double asum = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) asum = __dadd_rn(asum, ad[d]);
      if (s == 0) a0[0] = ad[0], a0[1] = ad[1], a0[2] = ad[2];
      // slot (s + 2) % 3 was last read before the previous barrier: cleared
      // for sub-step s + 2
      if (blockIdx.x == 0)
        for (int d = 0; d < 3; ++d) p.aslot[((s + 2) % 3) * 3 + d] = 0ull;
      // length of this sub-step: Eq. Time2 with its own alpha, the last one
      // ending exactly at the kinetic dt (same arithmetic in every block; the
      // quotient in the storage precision's arithmetic)
      double dtE = 0.0;
      int last = 0, bad = 0;
      if (g.forced_sub > 0) {
        dtE = g.dt / g.forced_sub;
        last = s + 1 == g.forced_sub;
      } else if (!(asum > 0.0)) {
        bad = 1;
      } else {
        const double cfl = sizeof(TF) == 8 ? __ddiv_rn(__dmul_rn(0.5, g.dx), asum)
                                           : (double)__fdiv_rn(0.5f * (float)g.dx, (float)asum);
        const double rem = __dsub_rn(g.dt, t);
        last = cfl >= rem;
        dtE = last ? rem : cfl;
      }
      s_dtE = dtE;
      s_k = sizeof(TF) == 8 ? (TF)(dtE / g.dx) : (TF)((float)dtE / (float)g.dx);
      for (int d = 0; d < 3; ++d) s_al[d] = (TF)ad[d];
      s_last = last;
      s_bad = bad;
      if (bad && blockIdx.x == 0) set_status(p.status, DVM_ERR_NONPHYSICAL);
    }
    __syncthreads();
    if (s_bad) return;
    const bool last = s_last != 0;
    const TF k = s_k;
    TF al[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) al[d] = s_al[d];
    TF amax[3] = {TF(0), TF(0), TF(0)};
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int x0 = (tile % ntx) * T::TX;
      const int y0 = ((tile / ntx) % nty) * T::TY;
      const int z = tile / (ntx * nty);
      if (tile != (int)blockIdx.x) {
        stage(src, tile);
        __syncthreads();
      }
      if (mydir == 0) tile_faces<TF, LIMITED, D, 0>(sw, sf, ctr, tx, ty, al[0]);
      else if (D >= 2 && mydir == 1) tile_faces<TF, LIMITED, D, (D >= 2 ? 1 : 0)>(sw, sf, ctr, tx, ty, al[D >= 2 ? 1 : 0]);
      else if (D == 3) tile_faces<TF, LIMITED, D, (D == 3 ? 2 : 0)>(sw, sf, ctr, tx, ty, al[D == 3 ? 2 : 0]);
      __syncthreads();
      const int gx = x0 + tx, gy = y0 + ty;
      if (mydir == 0 && gx < Nx && gy < Ny) {
        const int fbase = tx + T::FX * ty;
        const long long cell = gx + (long long)Nx * (gy + (long long)Ny * z);
        TF Wn[NM];
#pragma unroll
        for (int c = 0; c < NM; ++c) {
          TF acc = TF(0);
#pragma unroll
          for (int dir = 0; dir < D; ++dir) {
            const int fst = dir == 0 ? 1 : (dir == 1 ? T::FX : T::FX * T::FY);
            const TF* sfd = sf + (dir * NM + c) * T::NF;
            acc += sfd[fbase + fst] - sfd[fbase];
          }
          Wn[c] = sw[c * T::NS + ctr] - k * acc;
          dst[c * nc + cell] = Wn[c];
        }
        if (!last) {
          TF an[3];
          state_alpha_of<D>(Wn, an);
#pragma unroll
          for (int d = 0; d < 3; ++d) amax[d] = amax[d] > an[d] ? amax[d] : an[d];
        }
      }
      __syncthreads();
    }
    if (tid == 0) t = __dadd_rn(t, s_dtE);
    if (last) break;
    // merge this block's alpha of the new state into slot (s + 1) % 3 (the
    // bits of a non-negative double order like the value)
#pragma unroll
    for (int d = 0; d < D; ++d) {
      TF v = amax[d];
      for (int o = 16; o > 0; o >>= 1) {
        const TF w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
      }
      if ((tid & 31) == 0) s_amax[d][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < D) {
      TF v = TF(0);
      for (int w = 0; w < T::THREADS / 32; ++w) v = v > s_amax[tid][w] ? v : s_amax[tid][w];
      atomicMax(p.aslot + ((s + 1) % 3) * 3 + tid,
                (unsigned long long)__double_as_longlong((double)v));
    }
    if (s + 1 >= g.m_cap) {
      if (blockIdx.x == 0 && tid == 0) set_status(p.status, DVM_ERR_CFL);
      break;
    }
    if (!grid_sync(p.gbar, p.status)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    *p.msub = s + 1;
    for (int d = 0; d < 3; ++d) p.alpha[d] = a0[d];
  }
}

// ------------------------------------------------------------------ WENO5

// Interface value at j+1/2 from v[0..4] = the samples at j-2 .. j+2, biased
// to the left: the three third-order candidates of the sub-stencils
// {j-2, j-1, j}, {j-1, j, j+1}, {j, j+1, j+2} blended with the nonlinear
// weights d_k / (eps + beta_k)^2 (d = 1/10, 6/10, 3/10; beta_k the Jiang-Shu
// smoothness indicators; eps = 1e-6), normalised to one.
template <typename TF>
__device__ inline TF weno5_left(const TF v[5]) {
  const TF q0 = (TF(2) * v[0] - TF(7) * v[1] + TF(11) * v[2]) * TF(1.0 / 6.0);
  const TF q1 = (-v[1] + TF(5) * v[2] + TF(2) * v[3]) * TF(1.0 / 6.0);
  const TF q2 = (TF(2) * v[2] + TF(5) * v[3] - v[4]) * TF(1.0 / 6.0);
  const TF a0 = v[0] - TF(2) * v[1] + v[2], b0 = v[0] - TF(4) * v[1] + TF(3) * v[2];
  const TF a1 = v[1] - TF(2) * v[2] + v[3], b1 = v[1] - v[3];
  const TF a2 = v[2] - TF(2) * v[3] + v[4], b2 = TF(3) * v[2] - TF(4) * v[3] + v[4];
  const TF c13 = TF(13.0 / 12.0), eps = TF(1e-6);
  const TF e0 = eps + c13 * a0 * a0 + TF(0.25) * b0 * b0;
  const TF e1 = eps + c13 * a1 * a1 + TF(0.25) * b1 * b1;
  const TF e2 = eps + c13 * a2 * a2 + TF(0.25) * b2 * b2;
  const TF w0 = e_div(TF(0.1), e0 * e0), w1 = e_div(TF(0.6), e1 * e1), w2 = e_div(TF(0.3), e2 * e2);
  return e_div(w0 * q0 + w1 * q1 + w2 * q2, w0 + w1 + w2);
}

// -(psi_{j+1/2} - psi_{j-1/2}) along dir for one cell, from the cells j-3 ..
// j+3 of the state X (index list st[0..6]): the left-biased WENO5 value of
// f+ = (F + alpha U)/2 plus the right-biased (mirrored stencil) value of
// f- = (F - alpha U)/2 at each face.
template <typename TF, int D>
__device__ inline void weno_dir(const TF* X, long long nc, const long long st[7], int dir, TF al,
                                TF R[D + 2]) {
  constexpr int NM = D + 2;
  TF fp[7][NM], fm[7][NM];
#pragma unroll
  for (int o = 0; o < 7; ++o) {
    TF U[NM], F[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) U[i] = __ldcg(X + i * nc + st[o]);
    euler_flux<TF, D>(U, dir, F);
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      fp[o][i] = TF(0.5) * (F[i] + al * U[i]);
      fm[o][i] = TF(0.5) * (F[i] - al * U[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    TF psi[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {  // f = 0: face j-1/2 (cells j-3 .. j+2); f = 1: j+1/2
      const TF vp[5] = {fp[f][i], fp[f + 1][i], fp[f + 2][i], fp[f + 3][i], fp[f + 4][i]};
      const TF vm[5] = {fm[f + 5][i], fm[f + 4][i], fm[f + 3][i], fm[f + 2][i], fm[f + 1][i]};
      psi[f] = weno5_left<TF>(vp) + weno5_left<TF>(vm);
    }
    R[i] -= psi[1] - psi[0];
  }
}

// All Euler sub-steps of one kinetic step with the WENO5 solver (Section
// 4.3.3): per sub-step of Eq. Time2 length dt_E (alpha of its initial state,
// per direction, held for its three stages) the SSP Runge-Kutta stages
//   X1 = W + dt_E L(W),  X2 = 3/4 W + 1/4 (X1 + dt_E L(X1)),
//   W' = 1/3 W + 2/3 (X2 + dt_E L(X2)),  L = -(1/dx) sum_dir (psi+ - psi-),
// X1 and W' in the other ping-pong buffer, X2 in Wt; one cooperative launch,
// one thread per cell (grid-stride), a bounded grid barrier after each stage.
template <typename TF, int D>
__global__ void __launch_bounds__(kBlock) k_euler_weno(Geom g, DevPtrs p) {
  constexpr int NM = D + 2;
  __shared__ TF s_amax[3][kBlock / 32];
  __shared__ double s_dtE;
  __shared__ TF s_al[3];
  __shared__ int s_last, s_bad;
  const long long nc = g.nc;
  const int tid = threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  TF* Xt = (TF*)p.Wt;
  double t = 0.0, a0[3] = {0.0, 0.0, 0.0};
  // R = dt_E L(X) at cell c
  auto rhs = [&](const TF* X, long long c, const TF al[3], double dtE, TF R[NM]) {
    int x[3];
    cell_coords<D>(g, c, x);
#pragma unroll
    for (int i = 0; i < NM; ++i) R[i] = TF(0);
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
      long long st[7];
      int y[3] = {x[0], x[1], x[2]};
#pragma unroll
      for (int o = 0; o < 7; ++o) {
        y[dir] = bc_index(x[dir] + o - 3, g.nx[dir], g.bc[dir]);
        st[o] = cell_index(g, y);
      }
      weno_dir<TF, D>(X, nc, st, dir, al[dir], R);
    }
    const TF k = sizeof(TF) == 8 ? (TF)(dtE / g.dx) : (TF)((float)dtE / (float)g.dx);
#pragma unroll
    for (int i = 0; i < NM; ++i) R[i] *= k;
  };
  int s = 0;
  for (;; ++s) {
    const TF* W = (const TF*)((s & 1) ? p.W1 : p.W0);
    TF* X = (TF*)((s & 1) ? p.W0 : p.W1);
    if (tid == 0) {
      double ad[3], asum = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) ad[d] = __longlong_as_double((long long)__ldcg(p.aslot + (s % 3) * 3 + d));
#pragma unroll
      for (int d = 0; d < D; ++d) asum = __dadd_rn(asum, ad[d]);
      if (s == 0) a0[0] = ad[0], a0[1] = ad[1], a0[2] = ad[2];
      if (blockIdx.x == 0)
        for (int d = 0; d < 3; ++d) p.aslot[((s + 2) % 3) * 3 + d] = 0ull;
      double dtE = 0.0;
      int last = 0, bad = 0;
      if (g.forced_sub > 0) {
        dtE = g.dt / g.forced_sub;
        last = s + 1 == g.forced_sub;
      } else if (!(asum > 0.0)) {
        bad = 1;
      } else {
        const double cfl = sizeof(TF) == 8 ? __ddiv_rn(__dmul_rn(0.5, g.dx), asum)
                                           : (double)__fdiv_rn(0.5f * (float)g.dx, (float)asum);
        const double rem = __dsub_rn(g.dt, t);
        last = cfl >= rem;
        dtE = last ? rem : cfl;
      }
      s_dtE = dtE;
      for (int d = 0; d < 3; ++d) s_al[d] = (TF)ad[d];
      s_last = last;
      s_bad = bad;
      if (bad && blockIdx.x == 0) set_status(p.status, DVM_ERR_NONPHYSICAL);
    }
    __syncthreads();
    if (s_bad) return;
    const bool last = s_last != 0;
    const double dtE = s_dtE;
    const TF al[3] = {s_al[0], s_al[1], s_al[2]};
    TF R[NM];
    // stage 1: X = W + dt_E L(W)
    for (long long c = blockIdx.x * (long long)blockDim.x + tid; c < nc; c += stride) {
      rhs(W, c, al, dtE, R);
#pragma unroll
      for (int i = 0; i < NM; ++i) X[i * nc + c] = __ldcg(W + i * nc + c) + R[i];
    }
    if (!grid_sync(p.gbar, p.status)) return;
    // stage 2: Xt = 3/4 W + 1/4 (X + dt_E L(X))
    for (long long c = blockIdx.x * (long long)blockDim.x + tid; c < nc; c += stride) {
      rhs(X, c, al, dtE, R);
#pragma unroll
      for (int i = 0; i < NM; ++i)
        Xt[i * nc + c] = TF(0.75) * __ldcg(W + i * nc + c) + TF(0.25) * (__ldcg(X + i * nc + c) + R[i]);
    }
    if (!grid_sync(p.gbar, p.status)) return;
    // stage 3: X = 1/3 W + 2/3 (Xt + dt_E L(Xt)), and alpha of the new state
    TF amax[3] = {TF(0), TF(0), TF(0)};
    for (long long c = blockIdx.x * (long long)blockDim.x + tid; c < nc; c += stride) {
      rhs(Xt, c, al, dtE, R);
      TF Wn[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        Wn[i] = __ldcg(W + i * nc + c) * TF(1.0 / 3.0) + TF(2.0 / 3.0) * (__ldcg(Xt + i * nc + c) + R[i]);
        X[i * nc + c] = Wn[i];
      }
      if (!last) {
        TF an[3];
        state_alpha_of<D>(Wn, an);
#pragma unroll
        for (int d = 0; d < 3; ++d) amax[d] = amax[d] > an[d] ? amax[d] : an[d];
      }
    }
    if (tid == 0) t = __dadd_rn(t, dtE);
    if (last) break;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      TF v = amax[d];
      for (int o = 16; o > 0; o >>= 1) {
        const TF w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
      }
      if ((tid & 31) == 0) s_amax[d][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < D) {
      TF v = TF(0);
      for (int w = 0; w < kBlock / 32; ++w) v = v > s_amax[tid][w] ? v : s_amax[tid][w];
      atomicMax(p.aslot + ((s + 1) % 3) * 3 + tid, (unsigned long long)__double_as_longlong((double)v));
    }
    if (s + 1 >= g.m_cap) {
      if (blockIdx.x == 0 && tid == 0) set_status(p.status, DVM_ERR_CFL);
      break;
    }
    if (!grid_sync(p.gbar, p.status)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    *p.msub = s + 1;
    for (int d = 0; d < 3; ++d) p.alpha[d] = a0[d];
  }
}

// 1D and 2D Euler sub-steps with the split fluxes computed once per staged
// cell: after a tile and its halo are staged, G+ = F + alpha U and
// G- = F - alpha U of every staged cell and direction go to shared memory;
// each thread then computes one face flux (Eq. discmom with the van Leer
// slopes), psi_{j+1/2} = (G+_j + G-_{j+1}) / 2 + (sigma+_j - sigma-_{j+1}) / 4,
// which equals (F_j + F_{j+1}) / 2 - alpha (U_{j+1} - U_j) / 2 + (...) / 4.
template <int D, typename TF>
struct GTile {
  static constexpr int TX = D == 1 ? 128 : 32;
  static constexpr int TY = D == 1 ? 1 : 4;
  static constexpr int SX = TX + 4;
  static constexpr int SY = D >= 2 ? TY + 4 : 1;
  static constexpr int NS = SX * SY;
  static constexpr int FX = TX + 1, FY = D >= 2 ? TY + 1 : 1;
  static constexpr int NF = FX * FY;                  // face slots per direction
  static constexpr int NFX = (TX + 1) * TY;           // x faces of the tile
  static constexpr int NFY = D >= 2 ? TX * (TY + 1) : 0;
  static constexpr int CELLS = TX * TY;
  static constexpr int THREADS = ((NFX + NFY + 31) / 32) * 32;
  // staged W, G+/G- per direction, face fluxes per direction
  static constexpr size_t SMEM = (size_t)(D + 2) * (NS + 2 * D * NS + D * NF) * sizeof(TF);
};

template <typename TF, bool LIMITED, int D>
__device__ inline void face_from_g(const TF* __restrict__ sg, int c, int st, int dir, TF* __restrict__ sfd,
                                   int slot) {
  using T = GTile<D, TF>;
  constexpr int NM = D + 2;
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    const TF* gp = sg + ((dir * 2 + 0) * NM + i) * T::NS;
    const TF* gm = sg + ((dir * 2 + 1) * NM + i) * T::NS;
    const TF p0 = gp[c - st], p1 = gp[c], p2 = gp[c + st];
    const TF m1 = gm[c], m2 = gm[c + st], m3 = gm[c + 2 * st];
    const TF sp = slope<TF, LIMITED>(p1 - p0, p2 - p1);
    const TF sm = slope<TF, LIMITED>(m2 - m1, m3 - m2);
    sfd[i * T::NF + slot] = TF(0.5) * (p1 + m2) + TF(0.25) * (sp - sm);
  }
}

template <typename TF, bool LIMITED, int D>
__global__ void __launch_bounds__(GTile<D, TF>::THREADS, 4) k_euler_g(Geom g, DevPtrs p) {
  using T = GTile<D, TF>;
  constexpr int NM = D + 2;
  extern __shared__ unsigned char s_raw[];
  __shared__ TF s_amax[3][T::THREADS / 32];
  TF* sw = reinterpret_cast<TF*>(s_raw);  // [NM][SY][SX]
  TF* sg = sw + NM * T::NS;               // [D][2][NM][SY][SX]
  TF* sf = sg + 2 * D * NM * T::NS;       // [D][NM][FY][FX]
  const int Nx = g.nx[0], Ny = g.nx[1];
  const long long nc = g.nc;
  const int ntx = (Nx + T::TX - 1) / T::TX, nty = (Ny + T::TY - 1) / T::TY;
  const int ntiles = ntx * nty;
  const int tid = threadIdx.x;
  __shared__ double s_dtE;
  __shared__ TF s_k, s_al[3];
  __shared__ int s_last, s_bad;
  double t = 0.0, a0[3] = {0.0, 0.0, 0.0};
  auto stage = [&](const TF* src, int tile) {
    const int x0 = (tile % ntx) * T::TX;
    const int y0 = (tile / ntx) * T::TY;
    for (int i = tid; i < T::NS; i += T::THREADS) {
      const int lx = i % T::SX, ly = i / T::SX;
      const int gx = bc_index(x0 - 2 + lx, Nx, g.bc[0]);
      const int gy = D >= 2 ? bc_index(y0 - 2 + ly, Ny, g.bc[1]) : 0;
      const long long cc = gx + (long long)Nx * gy;
#pragma unroll
      for (int c = 0; c < NM; ++c) sw[c * T::NS + i] = __ldcg(src + c * nc + cc);
    }
  };
  int s = 0;
  for (;; ++s) {
    const TF* src = (const TF*)((s & 1) ? p.W1 : p.W0);
    TF* dst = (TF*)((s & 1) ? p.W0 : p.W1);
    double ad[3] = {0.0, 0.0, 0.0};
    if (tid == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) ad[d] = __longlong_as_double((long long)__ldcg(p.aslot + (s % 3) * 3 + d));
    }
    if ((int)blockIdx.x < ntiles) stage(src, blockIdx.x);
    if (tid == 0) {
      // alpha of this sub-step's initial state (slot s % 3); slot (s + 2) % 3
      // cleared for sub-step s + 2; the length of the sub-step by Eq. Time2,
      // the last one ending exactly at the kinetic dt
      double asum = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) asum = __dadd_rn(asum, ad[d]);
      if (s == 0) a0[0] = ad[0], a0[1] = ad[1], a0[2] = ad[2];
      if (blockIdx.x == 0)
        for (int d = 0; d < 3; ++d) p.aslot[((s + 2) % 3) * 3 + d] = 0ull;
      double dtE = 0.0;
      int last = 0, bad = 0;
      if (g.forced_sub > 0) {
        dtE = g.dt / g.forced_sub;
        last = s + 1 == g.forced_sub;
      } else if (!(asum > 0.0)) {
        bad = 1;
      } else {
        const double cfl = sizeof(TF) == 8 ? __ddiv_rn(__dmul_rn(0.5, g.dx), asum)
                                           : (double)__fdiv_rn(0.5f * (float)g.dx, (float)asum);
        const double rem = __dsub_rn(g.dt, t);
        last = cfl >= rem;
        dtE = last ? rem : cfl;
      }
      s_dtE = dtE;
      s_k = sizeof(TF) == 8 ? (TF)(dtE / g.dx) : (TF)((float)dtE / (float)g.dx);
      for (int d = 0; d < 3; ++d) s_al[d] = (TF)ad[d];
      s_last = last;
      s_bad = bad;
      if (bad && blockIdx.x == 0) set_status(p.status, DVM_ERR_NONPHYSICAL);
    }
    __syncthreads();
    if (s_bad) return;
    const bool last = s_last != 0;
    const TF k = s_k;
    TF al[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) al[d] = s_al[d];
    TF amax[3] = {TF(0), TF(0), TF(0)};
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int x0 = (tile % ntx) * T::TX;
      const int y0 = (tile / ntx) * T::TY;
      if (tile != (int)blockIdx.x) {
        stage(src, tile);
        __syncthreads();
      }
      // split fluxes of every staged cell and direction
      for (int i = tid; i < T::NS; i += T::THREADS) {
        TF U[NM], F[NM];
#pragma unroll
        for (int c = 0; c < NM; ++c) U[c] = sw[c * T::NS + i];
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
          euler_flux<TF, D>(U, dir, F);
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            sg[((dir * 2 + 0) * NM + c) * T::NS + i] = F[c] + al[dir] * U[c];
            sg[((dir * 2 + 1) * NM + c) * T::NS + i] = F[c] - al[dir] * U[c];
          }
        }
      }
      __syncthreads();
      // one face per thread: slot (fx, fy) is the low face of local cell (fx, fy)
      if (tid < T::NFX) {
        const int fx = tid % T::FX, fy = tid / T::FX;
        face_from_g<TF, LIMITED, D>(sg, fx + 1 + T::SX * (D >= 2 ? fy + 2 : 0), 1, 0, sf, fx + T::FX * fy);
      } else if (D >= 2 && tid < T::NFX + T::NFY) {
        const int f = tid - T::NFX;
        const int fx = f % T::TX, fy = f / T::TX;
        face_from_g<TF, LIMITED, D>(sg, fx + 2 + T::SX * (fy + 1), T::SX, D >= 2 ? 1 : 0,
                                    sf + (D >= 2 ? NM * T::NF : 0), fx + T::FX * fy);
      }
      __syncthreads();
      if (tid < T::CELLS) {
        const int tx = tid % T::TX, ty = tid / T::TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < Nx && gy < (D >= 2 ? Ny : 1)) {
          const int fbase = tx + T::FX * ty;
          const int ctr = tx + 2 + T::SX * (D >= 2 ? ty + 2 : 0);
          const long long cell = gx + (long long)Nx * gy;
          TF Wn[NM];
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            TF acc = TF(0);
#pragma unroll
            for (int dir = 0; dir < D; ++dir) {
              const int fst = dir == 0 ? 1 : T::FX;
              const TF* sfd = sf + (dir * NM + c) * T::NF;
              acc += sfd[fbase + fst] - sfd[fbase];
            }
            Wn[c] = sw[c * T::NS + ctr] - k * acc;
            dst[c * nc + cell] = Wn[c];
          }
          if (!last) {
            TF an[3];
            state_alpha_of<D>(Wn, an);
#pragma unroll
            for (int d = 0; d < 3; ++d) amax[d] = amax[d] > an[d] ? amax[d] : an[d];
          }
        }
      }
      __syncthreads();
    }
    if (tid == 0) t = __dadd_rn(t, s_dtE);
    if (last) break;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      TF v = amax[d];
      for (int o = 16; o > 0; o >>= 1) {
        const TF w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
      }
      if ((tid & 31) == 0) s_amax[d][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < D) {
      TF v = TF(0);
      for (int w = 0; w < T::THREADS / 32; ++w) v = v > s_amax[tid][w] ? v : s_amax[tid][w];
      atomicMax(p.aslot + ((s + 1) % 3) * 3 + tid, (unsigned long long)__double_as_longlong((double)v));
    }
    if (s + 1 >= g.m_cap) {
      if (blockIdx.x == 0 && tid == 0) set_status(p.status, DVM_ERR_CFL);
      break;
    }
    if (!grid_sync(p.gbar, p.status)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    *p.msub = s + 1;
    for (int d = 0; d < 3; ++d) p.alpha[d] = a0[d];
  }
}

// The same sub-steps in two phases per tile: (1) one thread per cell stages
// the tile and its halo (rounds over the staged cells) and computes the split
// fluxes of every staged cell it loaded, (2) every thread updates its own
// cell from the four (2D; two in 1D) faces it computes itself from the split
// fluxes.  Two block barriers per sub-step instead of four, every thread busy
// in both phases; the faces between two cells are computed twice.
//
// Tile shapes: 128 cells (1D), 32 x 4 (2D) and, for FP32 2D grids of at most
// one tile per two SMs, 32 x 32 ("tall"): a 1024-thread CTA takes 48K of an
// SM's 64K registers, so no CTA of the concurrent kinetic pass (32K) fits
// beside it and the Euler sub-steps run on SMs of their own while the kinetic
// pass keeps full occupancy on the others.  With 32 x 4 tiles (3-4 CTAs per
// SM) the block scheduler spreads them over every SM; each SM then also holds
// one kinetic CTA, and the Euler sub-steps, slowed by the kinetic pass's
// memory traffic on the same SMs, become the critical path of the step.
template <int D, typename TF, bool TALL = false>
struct G2Tile {
  static constexpr int TX = D == 1 ? 128 : 32;
  static constexpr int TY = D == 1 ? 1 : (TALL ? 32 : 4);
  static constexpr int SX = TX + 4;
  static constexpr int SY = D >= 2 ? TY + 4 : 1;
  static constexpr int NS = SX * SY;
  static constexpr int CELLS = TX * TY;
  static constexpr int THREADS = CELLS;
  static constexpr size_t SMEM = (size_t)(D + 2) * (NS + 2 * D * NS) * sizeof(TF);
};

// psi_{j+1/2} of component i along a direction from the split fluxes of the
// staged cells c - st .. c + 2 st (cell j at c)
template <typename TF, bool LIMITED>
__device__ inline TF face_g(const TF* __restrict__ gp, const TF* __restrict__ gm, int c, int st) {
  const TF p0 = gp[c - st], p1 = gp[c], p2 = gp[c + st];
  const TF m1 = gm[c], m2 = gm[c + st], m3 = gm[c + 2 * st];
  const TF sp = slope<TF, LIMITED>(p1 - p0, p2 - p1);
  const TF sm = slope<TF, LIMITED>(m2 - m1, m3 - m2);
  return TF(0.5) * (p1 + m2) + TF(0.25) * (sp - sm);
}

template <typename TF, bool LIMITED, int D, bool TALL>
__global__ void __launch_bounds__(G2Tile<D, TF, TALL>::THREADS) k_euler_g2(Geom g, DevPtrs p) {
  using T = G2Tile<D, TF, TALL>;
  constexpr int NM = D + 2;
  extern __shared__ unsigned char s_raw[];
  __shared__ TF s_amax[3][T::THREADS / 32];
  TF* sw = reinterpret_cast<TF*>(s_raw);  // [NM][SY][SX]
  TF* sg = sw + NM * T::NS;               // [D][2][NM][SY][SX]
  const int Nx = g.nx[0], Ny = g.nx[1];
  const long long nc = g.nc;
  const int ntx = (Nx + T::TX - 1) / T::TX, nty = (Ny + T::TY - 1) / T::TY;
  const int ntiles = ntx * nty;
  const int tid = threadIdx.x;
  __shared__ double s_dtE;
  __shared__ TF s_k, s_al[3];
  __shared__ int s_last, s_bad;
  double t = 0.0, a0[3] = {0.0, 0.0, 0.0};
  int s = 0;
  for (;; ++s) {
    const TF* src = (const TF*)((s & 1) ? p.W1 : p.W0);
    TF* dst = (TF*)((s & 1) ? p.W0 : p.W1);
    if (tid == 0) {
      double ad[3], asum = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) ad[d] = __longlong_as_double((long long)__ldcg(p.aslot + (s % 3) * 3 + d));
#pragma unroll
      for (int d = 0; d < D; ++d) asum = __dadd_rn(asum, ad[d]);
      if (s == 0) a0[0] = ad[0], a0[1] = ad[1], a0[2] = ad[2];
      if (blockIdx.x == 0)
        for (int d = 0; d < 3; ++d) p.aslot[((s + 2) % 3) * 3 + d] = 0ull;
      double dtE = 0.0;
      int last = 0, bad = 0;
      if (g.forced_sub > 0) {
        dtE = g.dt / g.forced_sub;
        last = s + 1 == g.forced_sub;
      } else if (!(asum > 0.0)) {
        bad = 1;
      } else {
        const double cfl = sizeof(TF) == 8 ? __ddiv_rn(__dmul_rn(0.5, g.dx), asum)
                                           : (double)__fdiv_rn(0.5f * (float)g.dx, (float)asum);
        const double rem = __dsub_rn(g.dt, t);
        last = cfl >= rem;
        dtE = last ? rem : cfl;
      }
      s_dtE = dtE;
      s_k = sizeof(TF) == 8 ? (TF)(dtE / g.dx) : (TF)((float)dtE / (float)g.dx);
      for (int d = 0; d < 3; ++d) s_al[d] = (TF)ad[d];
      s_last = last;
      s_bad = bad;
      if (bad && blockIdx.x == 0) set_status(p.status, DVM_ERR_NONPHYSICAL);
    }
    __syncthreads();
    if (s_bad) return;
    const bool last = s_last != 0;
    const TF k = s_k;
    TF al[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) al[d] = s_al[d];
    TF amax[3] = {TF(0), TF(0), TF(0)};
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int x0 = (tile % ntx) * T::TX;
      const int y0 = (tile / ntx) * T::TY;
      // phase 1: stage the tile and its two-cell halo, and the split fluxes
      // of every staged cell and direction
      for (int i = tid; i < T::NS; i += T::THREADS) {
        const int lx = i % T::SX, ly = i / T::SX;
        const int gx = bc_index(x0 - 2 + lx, Nx, g.bc[0]);
        const int gy = D >= 2 ? bc_index(y0 - 2 + ly, Ny, g.bc[1]) : 0;
        const long long cc = gx + (long long)Nx * gy;
        TF U[NM], F[NM];
#pragma unroll
        for (int c = 0; c < NM; ++c) {
          U[c] = __ldcg(src + c * nc + cc);
          sw[c * T::NS + i] = U[c];
        }
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
          euler_flux<TF, D>(U, dir, F);
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            sg[((dir * 2 + 0) * NM + c) * T::NS + i] = F[c] + al[dir] * U[c];
            sg[((dir * 2 + 1) * NM + c) * T::NS + i] = F[c] - al[dir] * U[c];
          }
        }
      }
      __syncthreads();
      // phase 2: every thread its cell, from its own faces
      const int tx = tid % T::TX, ty = tid / T::TX;
      const int gx = x0 + tx, gy = y0 + ty;
      if (gx < Nx && gy < (D >= 2 ? Ny : 1)) {
        const int ctr = tx + 2 + T::SX * (D >= 2 ? ty + 2 : 0);
        const long long cell = gx + (long long)Nx * gy;
        TF Wn[NM];
#pragma unroll
        for (int c = 0; c < NM; ++c) {
          TF acc = TF(0);
#pragma unroll
          for (int dir = 0; dir < D; ++dir) {
            const int st = dir == 0 ? 1 : T::SX;
            const TF* gp = sg + ((dir * 2 + 0) * NM + c) * T::NS;
            const TF* gm = sg + ((dir * 2 + 1) * NM + c) * T::NS;
            acc += face_g<TF, LIMITED>(gp, gm, ctr, st) - face_g<TF, LIMITED>(gp, gm, ctr - st, st);
          }
          Wn[c] = sw[c * T::NS + ctr] - k * acc;
          dst[c * nc + cell] = Wn[c];
        }
        if (!last) {
          TF an[3];
          state_alpha_of<D>(Wn, an);
#pragma unroll
          for (int d = 0; d < 3; ++d) amax[d] = amax[d] > an[d] ? amax[d] : an[d];
        }
      }
      __syncthreads();
    }
    if (tid == 0) t = __dadd_rn(t, s_dtE);
    if (last) break;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      TF v = amax[d];
      for (int o = 16; o > 0; o >>= 1) {
        const TF w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
      }
      if ((tid & 31) == 0) s_amax[d][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < D) {
      TF v = TF(0);
      for (int w = 0; w < T::THREADS / 32; ++w) v = v > s_amax[tid][w] ? v : s_amax[tid][w];
      atomicMax(p.aslot + ((s + 1) % 3) * 3 + tid, (unsigned long long)__double_as_longlong((double)v));
    }
    if (s + 1 >= g.m_cap) {
      if (blockIdx.x == 0 && tid == 0) set_status(p.status, DVM_ERR_CFL);
      break;
    }
    if (!grid_sync(p.gbar, p.status)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    *p.msub = s + 1;
    for (int d = 0; d < 3; ++d) p.alpha[d] = a0[d];
  }
}

// 3D sub-steps marching along z.  A CTA owns a 32 x 4 column of cells over a
// chunk of consecutive z planes.  Per plane it stages the plane's tile with its
// two-cell x/y halo (whose x and y split fluxes G+- = F +- alpha W it
// computes) and the tile's cells two planes ahead (their z split fluxes, kept
// in a ring of four planes), then computes every face flux once and updates
// each cell from its six faces.  A cell's state is read ~3.3 times per
// sub-step (plus four ring planes per chunk), against 11.25 with a 36 x 8 x 5
// staging per 32 x 4 x 1 tile.  Face fluxes as in k_euler_g2: psi = (G+_j +
// G-_{j+1}) / 2 + (s+ - s-) / 4; a warp is one tile row, so a lane's left x
// face is its left neighbour's right face (shuffled), the y faces go through
// shared memory, and a cell's lower z face is the upper face of the cell
// below, computed one plane earlier by the same thread.
template <typename TF>
struct ZTile {
  static constexpr int TX = 32, TY = 4, SX = TX + 4, SY = TY + 4;
  static constexpr int NS = SX * SY;     // staged plane cells
  static constexpr int CELLS = TX * TY;  // = threads
  static constexpr int THREADS = CELLS;
  static constexpr int NM = 5;
  static constexpr int RING = 4;
  // W of the plane, G+- along x and y of the plane, G+- along z of four
  // planes, the y face fluxes of the tile (TY + 1 rows)
  static constexpr size_t SMEM =
      sizeof(TF) * ((size_t)NM * NS + 4 * NM * NS + RING * 2 * NM * CELLS + NM * (TY + 1) * TX);
};

template <typename TF, bool LIMITED>
__device__ inline TF face6(TF p0, TF p1, TF p2, TF m1, TF m2, TF m3) {
  const TF sp = slope<TF, LIMITED>(p1 - p0, p2 - p1);
  const TF sm = slope<TF, LIMITED>(m2 - m1, m3 - m2);
  return TF(0.5) * (p1 + m2) + TF(0.25) * (sp - sm);
}

template <typename TF, bool LIMITED>
__global__ void __launch_bounds__(ZTile<TF>::THREADS) k_euler_z(Geom g, DevPtrs p) {
  using T = ZTile<TF>;
  constexpr int NM = 5;
  extern __shared__ unsigned char s_raw[];
  __shared__ TF s_amax[3][T::THREADS / 32];
  TF* sw = reinterpret_cast<TF*>(s_raw);  // [NM][NS]
  TF* sg = sw + NM * T::NS;               // [dir x/y][+-][NM][NS]
  TF* sz = sg + 4 * NM * T::NS;           // [ring 4][+-][NM][CELLS]
  TF* sfy = sz + T::RING * 2 * NM * T::CELLS;  // [NM][TY + 1][TX] y faces
  const int Nx = g.nx[0], Ny = g.nx[1], Nz = g.nx[2];
  const long long nc = g.nc, plane = (long long)Nx * Ny;
  const int ntx = (Nx + T::TX - 1) / T::TX, nty = (Ny + T::TY - 1) / T::TY;
  const int ntxy = ntx * nty;
  // z chunks: as many as the grid holds whole sets of column tiles
  int chunks = (int)gridDim.x / ntxy;
  chunks = chunks < 1 ? 1 : (chunks > Nz ? Nz : chunks);
  const int zc_len = (Nz + chunks - 1) / chunks;
  const int nitems = ntxy * chunks;
  const int tid = threadIdx.x;
  const int tx = tid % T::TX, ty = tid / T::TX;
  const int ctr = (tx + 2) + T::SX * (ty + 2);
  __shared__ double s_dtE;
  __shared__ TF s_k, s_al[3];
  __shared__ int s_last, s_bad;
  double t = 0.0, a0[3] = {0.0, 0.0, 0.0};
  int s = 0;
  for (;; ++s) {
    const TF* src = (const TF*)((s & 1) ? p.W1 : p.W0);
    TF* dst = (TF*)((s & 1) ? p.W0 : p.W1);
    if (tid == 0) {
      double ad[3], asum = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) ad[d] = __longlong_as_double((long long)__ldcg(p.aslot + (s % 3) * 3 + d));
#pragma unroll
      for (int d = 0; d < 3; ++d) asum = __dadd_rn(asum, ad[d]);
      if (s == 0) a0[0] = ad[0], a0[1] = ad[1], a0[2] = ad[2];
      if (blockIdx.x == 0)
        for (int d = 0; d < 3; ++d) p.aslot[((s + 2) % 3) * 3 + d] = 0ull;
      double dtE = 0.0;
      int last = 0, bad = 0;
      if (g.forced_sub > 0) {
        dtE = g.dt / g.forced_sub;
        last = s + 1 == g.forced_sub;
      } else if (!(asum > 0.0)) {
        bad = 1;
      } else {
        const double cfl = sizeof(TF) == 8 ? __ddiv_rn(__dmul_rn(0.5, g.dx), asum)
                                           : (double)__fdiv_rn(0.5f * (float)g.dx, (float)asum);
        const double rem = __dsub_rn(g.dt, t);
        last = cfl >= rem;
        dtE = last ? rem : cfl;
      }
      s_dtE = dtE;
      s_k = sizeof(TF) == 8 ? (TF)(dtE / g.dx) : (TF)((float)dtE / (float)g.dx);
      for (int d = 0; d < 3; ++d) s_al[d] = (TF)ad[d];
      s_last = last;
      s_bad = bad;
      if (bad && blockIdx.x == 0) set_status(p.status, DVM_ERR_NONPHYSICAL);
    }
    __syncthreads();
    if (s_bad) return;
    const bool last = s_last != 0;
    const TF k = s_k;
    const TF al0 = s_al[0], al1 = s_al[1], al2 = s_al[2];
    TF amax[3] = {TF(0), TF(0), TF(0)};
    // z split fluxes of the tile's cells on plane zz into ring slot zz mod 4
    auto ring = [&](int zz) { return sz + ((zz + 2 * T::RING) % T::RING) * 2 * NM * T::CELLS; };
    auto ring_cell = [&](int x0, int y0, int zz) {
      const int gx = bc_index(x0 + tx, Nx, g.bc[0]);
      const int gy = bc_index(y0 + ty, Ny, g.bc[1]);
      const int gz = bc_index(zz, Nz, g.bc[2]);
      return gx + (long long)Nx * gy + plane * gz;
    };
    // from the state U of the thread's cell on plane zz
    auto ring_store = [&](int zz, const TF* U) {
      TF F[NM];
      euler_flux<TF, 3>(U, 2, F);
      TF* r = ring(zz);
#pragma unroll
      for (int c = 0; c < NM; ++c) {
        r[c * T::CELLS + tid] = F[c] + al2 * U[c];
        r[(NM + c) * T::CELLS + tid] = F[c] - al2 * U[c];
      }
    };
    auto ring_plane = [&](int x0, int y0, int zz) {
      const long long cc = ring_cell(x0, y0, zz);
      TF U[NM];
#pragma unroll
      for (int c = 0; c < NM; ++c) U[c] = __ldcg(src + c * nc + cc);
      ring_store(zz, U);
    };
    // the states phase 1 of plane zz reads (the thread's staged cells i = tid,
    // tid + 128, tid + 256 and its cell two planes ahead), loaded one plane
    // early so that their L2 round trip overlaps the previous plane's faces
    constexpr int KS = (T::NS + T::THREADS - 1) / T::THREADS;
    TF pre[KS][NM], pre_r[NM];
    auto prefetch = [&](int x0, int y0, int zz) {
      const int gz = bc_index(zz, Nz, g.bc[2]);
#pragma unroll
      for (int q = 0; q < KS; ++q) {
        const int i = tid + q * T::THREADS;
        if (i < T::NS) {
          const int lx = i % T::SX, ly = i / T::SX;
          const int gx = bc_index(x0 - 2 + lx, Nx, g.bc[0]);
          const int gy = bc_index(y0 - 2 + ly, Ny, g.bc[1]);
          const long long cc = gx + (long long)Nx * gy + plane * gz;
#pragma unroll
          for (int c = 0; c < NM; ++c) pre[q][c] = __ldcg(src + c * nc + cc);
        }
      }
      const long long cr = ring_cell(x0, y0, zz + 2);
#pragma unroll
      for (int c = 0; c < NM; ++c) pre_r[c] = __ldcg(src + c * nc + cr);
    };
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      const int txy = item % ntxy, chunk = item / ntxy;
      const int x0 = (txy % ntx) * T::TX, y0 = (txy / ntx) * T::TY;
      const int z0 = chunk * zc_len;
      const int z1 = z0 + zc_len < Nz ? z0 + zc_len : Nz;
      if (z0 >= z1) continue;
      for (int zz = z0 - 2; zz < z0 + 2; ++zz) ring_plane(x0, y0, zz);
      // the face below the first plane (between z0 - 1 and z0); each thread
      // reads only its own column of the ring
      TF fzl[NM];
      {
        const TF *rm2 = ring(z0 - 2), *rm1 = ring(z0 - 1), *r0 = ring(z0), *r1 = ring(z0 + 1);
#pragma unroll
        for (int c = 0; c < NM; ++c) {
          const int op = c * T::CELLS + tid, om = (NM + c) * T::CELLS + tid;
          fzl[c] = face6<TF, LIMITED>(rm2[op], rm1[op], r0[op], rm1[om], r0[om], r1[om]);
        }
      }
      prefetch(x0, y0, z0);
      for (int zc = z0; zc < z1; ++zc) {
        // phase 1: the plane's tile and halo with its x and y split fluxes,
        // and the z split fluxes two planes ahead
#pragma unroll
        for (int q = 0; q < KS; ++q) {
          const int i = tid + q * T::THREADS;
          if (i >= T::NS) continue;
          TF U[NM], F[NM];
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            U[c] = pre[q][c];
            sw[c * T::NS + i] = U[c];
          }
          euler_flux<TF, 3>(U, 0, F);
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            sg[(0 * NM + c) * T::NS + i] = F[c] + al0 * U[c];
            sg[(1 * NM + c) * T::NS + i] = F[c] - al0 * U[c];
          }
          euler_flux<TF, 3>(U, 1, F);
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            sg[(2 * NM + c) * T::NS + i] = F[c] + al1 * U[c];
            sg[(3 * NM + c) * T::NS + i] = F[c] - al1 * U[c];
          }
        }
        ring_store(zc + 2, pre_r);
        if (zc + 1 < z1) prefetch(x0, y0, zc + 1);
        __syncthreads();
        // phase 2: every face flux once.  x: lane tx its right face, the
        // row's left boundary face from lanes 0..NM-1 (component = lane).
        // y: every thread its upper face, the tile's lower boundary faces
        // shared out, all into sfy.  z: the face above the plane.
        TF fxr[NM], fxl[NM], fyt[NM], fzh[NM];
        {
          TF fb = TF(0);
          if (tx < NM)
            fb = face_g<TF, LIMITED>(sg + (0 * NM + tx) * T::NS, sg + (1 * NM + tx) * T::NS, ctr - tx - 1, 1);
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            fxr[c] = face_g<TF, LIMITED>(sg + (0 * NM + c) * T::NS, sg + (1 * NM + c) * T::NS, ctr, 1);
            const TF up = __shfl_up_sync(0xffffffffu, fxr[c], 1);
            const TF bnd = __shfl_sync(0xffffffffu, fb, c);
            fxl[c] = tx == 0 ? bnd : up;
          }
        }
#pragma unroll
        for (int c = 0; c < NM; ++c) {
          fyt[c] = face_g<TF, LIMITED>(sg + (2 * NM + c) * T::NS, sg + (3 * NM + c) * T::NS, ctr, T::SX);
          sfy[(c * (T::TY + 1) + ty + 1) * T::TX + tx] = fyt[c];
        }
        for (int i = tid; i < NM * T::TX; i += T::THREADS) {
          const int c = i / T::TX, xx = i % T::TX;
          sfy[(c * (T::TY + 1)) * T::TX + xx] = face_g<TF, LIMITED>(
              sg + (2 * NM + c) * T::NS, sg + (3 * NM + c) * T::NS, (xx + 2) + T::SX, T::SX);
        }
        {
          const TF *rm1 = ring(zc - 1), *r0 = ring(zc), *r1 = ring(zc + 1), *r2 = ring(zc + 2);
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            const int op = c * T::CELLS + tid, om = (NM + c) * T::CELLS + tid;
            fzh[c] = face6<TF, LIMITED>(rm1[op], r0[op], r1[op], r0[om], r1[om], r2[om]);
          }
        }
        __syncthreads();
        // phase 3: every thread its cell, from its six faces
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < Nx && gy < Ny) {
          const long long cell = gx + (long long)Nx * gy + plane * zc;
          TF Wn[NM];
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            TF acc = fxr[c] - fxl[c];
            acc += fyt[c] - sfy[(c * (T::TY + 1) + ty) * T::TX + tx];
            acc += fzh[c] - fzl[c];
            Wn[c] = sw[c * T::NS + ctr] - k * acc;
            dst[c * nc + cell] = Wn[c];
          }
          if (!last) {
            TF an[3];
            state_alpha_of<3>(Wn, an);
#pragma unroll
            for (int d = 0; d < 3; ++d) amax[d] = amax[d] > an[d] ? amax[d] : an[d];
          }
        }
#pragma unroll
        for (int c = 0; c < NM; ++c) fzl[c] = fzh[c];
        __syncthreads();
      }
    }
    if (tid == 0) t = __dadd_rn(t, s_dtE);
    if (last) break;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      TF v = amax[d];
      for (int o = 16; o > 0; o >>= 1) {
        const TF w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
      }
      if ((tid & 31) == 0) s_amax[d][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < 3) {
      TF v = TF(0);
      for (int w = 0; w < T::THREADS / 32; ++w) v = v > s_amax[tid][w] ? v : s_amax[tid][w];
      atomicMax(p.aslot + ((s + 1) % 3) * 3 + tid, (unsigned long long)__double_as_longlong((double)v));
    }
    if (s + 1 >= g.m_cap) {
      if (blockIdx.x == 0 && tid == 0) set_status(p.status, DVM_ERR_CFL);
      break;
    }
    if (!grid_sync(p.gbar, p.status)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    *p.msub = s + 1;
    for (int d = 0; d < 3; ++d) p.alpha[d] = a0[d];
  }
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
// (Eq. minim_full), checks, the parameters of the next pass, and for HOFKS
// alpha, W = (1 - lambda) U^{n+1} and the sub-step count of the next step.
template <typename TC, typename TW, int SCHEME, int D>
__global__ void __launch_bounds__(kBlock) k_finalize(Geom g, DevPtrs p) {
  constexpr int NM = D + 2;
  constexpr bool HO = SCHEME != DVM_FKS;
  constexpr int NACC = HO ? 2 * NM : NM;
  // FP32-storage builds: moments combined in FP64 (the partial sums, U^{n+1}
  // = U_* + U_E, U_E - U_M, U - C M[U]), the rest of the per-cell arithmetic
  // in FP32 (GB300's FP64 rate bounds this kernel otherwise)
  constexpr bool F32 = sizeof(TC) == 4;
  using TA = typename std::conditional<F32, float, double>::type;
  __shared__ float sA[kMaxM * kMaxM];
  if (F32) stage_af<D>(p, sA);
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c == 0) *p.step += 1;
  const long long nc = g.nc;
  TA a[3] = {0, 0, 0};
  if (c < nc) {
    double Un[kMaxM], r[kMaxM] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double sums[2 * kMaxM];
#pragma unroll
    for (int j = 0; j < NACC; ++j) {
      double s = 0.0;
      for (int sp = 0; sp < g.nsplit; ++sp) s += p.acc[((long long)sp * 2 * NM + j) * nc + c];
      sums[j] = g.w * s;
    }
    if (HO) {
      const TW* UE = (const TW*)((*p.msub & 1) ? p.W1 : p.W0);
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        const double ue = g.skip_euler ? 0.0 : (double)UE[i * nc + c];
        r[i] = ue - sums[NM + i];
        Un[i] = sums[i] + ue;
        p.UE[i * nc + c] = ue;
        p.Us[i * nc + c] = sums[i];
        p.UM[i * nc + c] = sums[NM + i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        Un[i] = sums[i];
        p.Us[i * nc + c] = sums[i];
      }
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) p.U[i * nc + c] = Un[i];
    // the HOFKS correction nu = A (U_E - U_M); a flagged cell of the learned
    // path has f^{n+1} = E[U^{n+1}], no correction
    const bool no_nu = !HO || (g.learn && p.lflag[c]);
    const double lam = p.lam[c];
    int rc;
    if constexpr (F32) {
      float nu[kMaxM], mu[kMaxM], rho, u[3], theta;
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < NM; ++j) s = fmaf(sA[i * NM + j], (float)r[j], s);
        nu[i] = no_nu ? 0.f : s;
      }
      rc = cell_mu_f32<D>(g, sA, Un, mu, rho, u, theta);
      if (!rc) write_params_f32<D>(g, (float*)p.prm, c, (float)lam, (float)(1.0 - lam), rho, u, theta,
                                   HO ? nu : nullptr, mu);
    } else {
      double nu[kMaxM], mu[kMaxM], rho, u[3], theta;
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NM; ++j) s += p.A[i * NM + j] * r[j];
        nu[i] = no_nu ? 0.0 : s;
      }
      rc = cell_mu<D>(g, p.A, Un, mu, rho, u, theta);
      if (!rc) write_params<TC, D>(g, (TC*)p.prm, c, lam, 1.0 - lam, rho, u, theta, HO ? nu : nullptr, mu);
    }
    if (rc) {
      set_status(p.status, rc);
    } else if (HO) {
      TW W[kMaxM];
      const double w = 1.0 - lam;
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        W[i] = (TW)(w * Un[i]);
        ((TW*)p.W0)[i * nc + c] = W[i];
      }
      state_alpha_of<D>(W, a);
    }
  }
  if (HO) alpha_reduce_publish<D, TA>(g, p, a);
}

// f at the cell centres: stored piece value plus the deferred term.
template <typename TS, typename TC, int D>
__global__ void k_materialize(Geom g, DevPtrs p, double* out) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.nc * g.nvel) return;
  const long long c = idx % g.nc, k = idx / g.nc;
  const long long n = *p.step, nc = g.nc;
  const TC* prm = (const TC*)p.prm;
  int x[3];
  const int kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
                     (int)(k / ((long long)g.nv[0] * g.nv[1]))};
  cell_coords<D>(g, c, x);
  int q[3] = {0, 0, 0};
  double v[3] = {0.0, 0.0, 0.0}, vv = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const long long kg = g.kmin[i] + kk[i];
    q[i] = wrap((long long)x[i] - transport_offset(kg, n, g.p), g.nx[i]);
    v[i] = (double)kg * g.dv;
    vv += v[i] * v[i];
  }
  const long long slot = cell_index(g, q);
  if (g.learn && p.lflag[c]) {
    // flagged in the last step: f = E[U] (weight-1 Maxwellian and mu)
    double qq = 0.0, lin = (double)prm[prm_at(row_mu(D, 0), c, nc)];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double du = v[i] - (double)prm[prm_at(row_u(i), c, nc)];
      qq += du * du;
      lin += (double)prm[prm_at(row_mu(D, 1 + i), c, nc)] * v[i];
    }
    lin += (double)prm[prm_at(row_mu(D, D + 1), c, nc)] * vv;
    const double e = (double)prm[prm_at(row_L(), c, nc)] - (double)prm[prm_at(row_h(D), c, nc)] * qq;
    out[k * nc + c] = (exp2(e) + lin) * p.linvw[c];
    return;
  }
  double f = (double)StoreT<TS>::load((const TS*)p.F + k * nc + slot);
  if (g.scheme == DVM_FKS) {
    double qq = 0.0, lin = (double)prm[prm_at(row_mu(D, 0), c, nc)];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double du = v[i] - (double)prm[prm_at(row_u(i), c, nc)];
      qq += du * du;
      lin += (double)prm[prm_at(row_mu(D, 1 + i), c, nc)] * v[i];
    }
    lin += (double)prm[prm_at(row_mu(D, D + 1), c, nc)] * vv;
    // the deferred equilibrium part (1 - lambda) E[U] (zero before the first step)
    const double def =
        exp2((double)prm[prm_at(row_L(), c, nc)] - (double)prm[prm_at(row_h(D), c, nc)] * qq) + lin;
    if (g.strang && n > 0) {
      // Strang splitting: the state is R_h T (R T)^(n-1) f^0, one half
      // relaxation short of the first-order R T (R T)^(n-1) f^0 kept here
      // (f_L - E = lambda_h (f_S - E), lambda_h^2 = lambda):
      // f_S = F / lambda_h + (1 - lambda) E / (1 + lambda_h)
      const double lh = sqrt(p.lam[c]);
      f = (lh > 0.0 ? f / lh : 0.0) + def / (1.0 + lh);
    } else {
      f += def;
    }
  } else {
    double lin = (double)prm[prm_at(row_nu(D, 0), c, nc)];
#pragma unroll
    for (int i = 0; i < D; ++i) lin += (double)prm[prm_at(row_nu(D, 1 + i), c, nc)] * v[i];
    lin += (double)prm[prm_at(row_nu(D, D + 1), c, nc)] * vv;
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

// Dispatch on the run-time dimension: CALL sees the constant DD.
#define DVM_BY_DIM(g, CALL)    \
  do {                         \
    if ((g).d == 1) {          \
      constexpr int DD = 1;    \
      CALL;                    \
    } else if ((g).d == 2) {   \
      constexpr int DD = 2;    \
      CALL;                    \
    } else {                   \
      constexpr int DD = 3;    \
      CALL;                    \
    }                          \
  } while (0)

template <typename TF, bool LIM, int D>
cudaError_t launch_euler_g(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare, int* blocks) {
  using T = GTile<D, TF>;
  if (prepare) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_euler_g<TF, LIM, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_g<TF, LIM, D>, T::THREADS, T::SMEM);
    const long long nb = (long long)sms * (per_sm < 1 ? 1 : per_sm);
    const long long need = (long long)((g.nx[0] + T::TX - 1) / T::TX) * ((g.nx[1] + T::TY - 1) / T::TY);
    *blocks = (int)(nb < need ? nb : need);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.euler_blocks);
  cfg.blockDim = dim3(T::THREADS);
  cfg.dynamicSmemBytes = T::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_euler_g<TF, LIM, D>, g, p);
}

template <typename TF, int D>
cudaError_t launch_euler_weno(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare, int* blocks) {
  if (prepare) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_weno<TF, D>, kBlock, 0);
    const long long nb = (long long)sms * (per_sm < 1 ? 1 : per_sm);
    const long long need = (g.nc + kBlock - 1) / kBlock;
    *blocks = (int)(nb < need ? nb : need);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.euler_blocks);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_euler_weno<TF, D>, g, p);
}

template <typename TF, bool LIM, int D, bool TALL>
cudaError_t launch_euler_g2_t(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare, int* blocks) {
  using T = G2Tile<D, TF, TALL>;
  if (prepare) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_euler_g2<TF, LIM, D, TALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_g2<TF, LIM, D, TALL>, T::THREADS, T::SMEM);
    const long long nb = (long long)sms * (per_sm < 1 ? 1 : per_sm);
    const long long need = (long long)((g.nx[0] + T::TX - 1) / T::TX) * ((g.nx[1] + T::TY - 1) / T::TY);
    *blocks = (int)(nb < need ? nb : need);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.euler_blocks);
  cfg.blockDim = dim3(T::THREADS);
  cfg.dynamicSmemBytes = T::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_euler_g2<TF, LIM, D, TALL>, g, p);
}

// 32 x 32 tiles: FP32 2D grids of at most one such tile per two SMs
// (DVM_EULER_TALL=0 keeps the 32 x 4 tiles, for comparison runs)
bool euler_tall(const Geom& g) {
  if (g.d != 2 || g.precision == DVM_F64) return false;
  const char* e = getenv("DVM_EULER_TALL");
  if (e && e[0] == '0') return false;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return false;
  const long long tiles = (long long)((g.nx[0] + 31) / 32) * ((g.nx[1] + 31) / 32);
  return 2 * tiles <= sms;
}

template <typename TF, bool LIM, int D>
cudaError_t launch_euler_g2(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare, int* blocks) {
  if constexpr (D == 2 && sizeof(TF) == 4)
    if (euler_tall(g)) return launch_euler_g2_t<TF, LIM, D, true>(g, p, s, prepare, blocks);
  return launch_euler_g2_t<TF, LIM, D, false>(g, p, s, prepare, blocks);
}

template <typename TF, bool LIM>
cudaError_t launch_euler_z(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare, int* blocks) {
  using T = ZTile<TF>;
  if (prepare) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_euler_z<TF, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_z<TF, LIM>, T::THREADS, T::SMEM);
    const long long nb = (long long)sms * (per_sm < 1 ? 1 : per_sm);
    // one work item per (column tile, z plane) at most
    const long long need = (long long)((g.nx[0] + T::TX - 1) / T::TX) * ((g.nx[1] + T::TY - 1) / T::TY) * g.nx[2];
    *blocks = (int)(nb < need ? nb : need);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.euler_blocks);
  cfg.blockDim = dim3(T::THREADS);
  cfg.dynamicSmemBytes = T::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_euler_z<TF, LIM>, g, p);
}

template <typename TF, bool LIM, int D>
cudaError_t launch_euler_t(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare,
                           int* blocks) {
  // DVM_EULER_KERNEL: 1 the per-face-flux kernel, 2 (1D/2D) the four-phase
  // split-flux kernel (comparison runs); default the two-phase one (1D/2D)
  // and the z-marching one (3D)
  const char* e = getenv("DVM_EULER_KERNEL");
  if constexpr (D <= 2) {
    if (e && e[0] == '2') return launch_euler_g<TF, LIM, D>(g, p, s, prepare, blocks);
    if (!(e && e[0] == '1')) return launch_euler_g2<TF, LIM, D>(g, p, s, prepare, blocks);
  } else {
    if (!(e && e[0] == '1')) return launch_euler_z<TF, LIM>(g, p, s, prepare, blocks);
  }
  using T = ETile<D, TF>;
  if (prepare) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_euler<TF, LIM, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)T::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler<TF, LIM, D>, T::THREADS, T::SMEM);
    const long long nb = (long long)sms * (per_sm < 1 ? 1 : per_sm);
    const long long need = (long long)((g.nx[0] + T::TX - 1) / T::TX) *
                           ((g.nx[1] + T::TY - 1) / T::TY) * g.nx[2];
    *blocks = (int)(nb < need ? nb : need);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.euler_blocks);
  cfg.blockDim = dim3(T::THREADS);
  cfg.dynamicSmemBytes = T::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_euler<TF, LIM, D>, g, p);
}

cudaError_t euler_dispatch(const Geom& g, const DevPtrs& p, cudaStream_t s, bool prepare,
                           int* blocks) {
  const bool lim = g.scheme == DVM_HOFKS;
  cudaError_t e = cudaSuccess;
  if (g.scheme == DVM_HOFKS_WENO) {
    if (g.precision == DVM_F64) DVM_BY_DIM(g, e = (launch_euler_weno<double, DD>(g, p, s, prepare, blocks)));
    else DVM_BY_DIM(g, e = (launch_euler_weno<float, DD>(g, p, s, prepare, blocks)));
    return e;
  }
  if (g.precision == DVM_F64) {
    if (lim) DVM_BY_DIM(g, e = (launch_euler_t<double, true, DD>(g, p, s, prepare, blocks)));
    else DVM_BY_DIM(g, e = (launch_euler_t<double, false, DD>(g, p, s, prepare, blocks)));
  } else {
    if (lim) DVM_BY_DIM(g, e = (launch_euler_t<float, true, DD>(g, p, s, prepare, blocks)));
    else DVM_BY_DIM(g, e = (launch_euler_t<float, false, DD>(g, p, s, prepare, blocks)));
  }
  return e;
}

}  // namespace

// ------------------------------------------------------------ launchers

void launch_prim_to_cons(const Geom& g, const double* rho, const double* u, const double* T,
                         double* U, cudaStream_t s) {
  DVM_BY_DIM(g, (k_prim_to_cons<DD><<<blocks_for(g.nc), kBlock, 0, s>>>(g, rho, u, T, U)));
}

void launch_cell_params(const Geom& g, const DevPtrs& p, int mode, int initial, cudaStream_t s) {
  if (g.precision == DVM_F64)
    DVM_BY_DIM(g, (k_cell_params<double, DD><<<blocks_for(g.nc), kBlock, 0, s>>>(g, p, mode, initial)));
  else
    DVM_BY_DIM(g, (k_cell_params<float, DD><<<blocks_for(g.nc), kBlock, 0, s>>>(g, p, mode, initial)));
}

void launch_init_f(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  if (g.precision == DVM_F64) {
    const unsigned nb = blocks_for(g.nc * g.nvel);
    DVM_BY_DIM(g, (k_init_f<double, DD><<<nb, kBlock, 0, s>>>(g, p)));
    return;
  }
  // FP32 / BF16: per-cell threads over velocity chunks of about 64 rows
  // (at least a few waves of CTAs on 152 SMs for small grids)
  const long long cb = blocks_for(g.nc);
  long long chunks = (g.nvel + 63) / 64;
  if (chunks > 65535) chunks = 65535;  // grid y limit
  const int kchunk = (int)((g.nvel + chunks - 1) / chunks);
  chunks = (g.nvel + kchunk - 1) / kchunk;
  const dim3 grid((unsigned)cb, (unsigned)chunks);
  if (g.precision == DVM_F32)
    DVM_BY_DIM(g, (k_init_f_rows<float, DD><<<grid, kBlock, 0, s>>>(g, p, kchunk)));
  else
    DVM_BY_DIM(g, (k_init_f_rows<__nv_bfloat16, DD><<<grid, kBlock, 0, s>>>(g, p, kchunk)));
}

void launch_alpha(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  if (g.precision == DVM_F64)
    DVM_BY_DIM(g, (k_alpha<double, DD><<<blocks_for(g.nc), kBlock, 0, s>>>(g, p)));
  else
    DVM_BY_DIM(g, (k_alpha<float, DD><<<blocks_for(g.nc), kBlock, 0, s>>>(g, p)));
}

int euler_blocks(const Geom& g) {
  int blocks = 1;
  euler_dispatch(g, DevPtrs{}, nullptr, true, &blocks);
  // DVM_EULER_BLOCKS caps the cooperative grid (launch-shape sweeps)
  const char* e = getenv("DVM_EULER_BLOCKS");
  if (e) {
    const int cap = atoi(e);
    if (cap > 0 && cap < blocks) blocks = cap;
  }
  return blocks < 1 ? 1 : blocks;
}

cudaError_t launch_euler(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  return euler_dispatch(g, p, s, false, nullptr);
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
  if (g.precision == DVM_F64) {
    if (g.scheme == DVM_FKS)
      DVM_BY_DIM(g, (k_finalize<double, double, DVM_FKS, DD><<<nb, kBlock, 0, s>>>(g, p)));
    else
      DVM_BY_DIM(g, (k_finalize<double, double, DVM_HOFKS, DD><<<nb, kBlock, 0, s>>>(g, p)));
  } else {
    if (g.scheme == DVM_FKS)
      DVM_BY_DIM(g, (k_finalize<float, float, DVM_FKS, DD><<<nb, kBlock, 0, s>>>(g, p)));
    else
      DVM_BY_DIM(g, (k_finalize<float, float, DVM_HOFKS, DD><<<nb, kBlock, 0, s>>>(g, p)));
  }
}

void launch_materialize(const Geom& g, const DevPtrs& p, double* out, cudaStream_t s) {
  const unsigned nb = blocks_for(g.nc * g.nvel);
  if (g.precision == DVM_F64)
    DVM_BY_DIM(g, (k_materialize<double, double, DD><<<nb, kBlock, 0, s>>>(g, p, out)));
  else if (g.precision == DVM_F32)
    DVM_BY_DIM(g, (k_materialize<float, float, DD><<<nb, kBlock, 0, s>>>(g, p, out)));
  else
    DVM_BY_DIM(g, (k_materialize<__nv_bfloat16, float, DD><<<nb, kBlock, 0, s>>>(g, p, out)));
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
// Fixed header: the status word at 0, the largest (C C^T)^{-1} (kMaxM^2
// doubles) from kNoAllocA, and the per-cell parameters from the next 256-byte
// boundary after it.  The three regions must not overlap: the parameter
// kernel writes cell 0's rows while other blocks still read the matrix.
constexpr size_t kNoAllocA = 64;
constexpr size_t kNoAllocHeader = DVM_NOALLOC_HEADER_BYTES;
static_assert(kNoAllocA + sizeof(double) * kMaxM * kMaxM <= kNoAllocHeader,
              "(C C^T)^{-1} must end before the per-cell parameters start");
static_assert(kNoAllocHeader % 256 == 0, "per-cell parameters start on a 256-byte boundary");

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
  // scratch layout: the status word at 0, (C C^T)^{-1} from kNoAllocA; the
  // equilibrium parameters (prm_rows x Nc) from kNoAllocHeader; then Nc
  // doubles read as lambda
  const size_t nc = (size_t)g.nc;
  const size_t need = kNoAllocHeader + 8 * (size_t)prm_rows(g.d) * nc + 8 * nc;
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
  p.A = (double*)(b + kNoAllocA);
  p.eqp = (double*)(b + kNoAllocHeader);
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
