// dvm_batch.cu -- many independent 1D-1V and 2D-2V cases advanced together.
//
// Cases differ in dimension, N_x (N_y), N_v, tau, p and boundary rule and
// share the scheme and the storage precision.  One time step of the whole
// batch is four launches, captured once into a CUDA graph:
//   k_b_prepare  the boundary pieces of outflow cases; reset of the work queue.
//   k_b_euler    one CTA per case (largest first), on a forked stream beside
//                the kinetic pass: alpha, W = (1 - lambda) U, all MUSCL
//                sub-steps (Section 4.3.2; a 1D tube in shared memory, a 2D
//                case unsplit in global memory), U_E.
//   k_b_kinetic  persistent: CTAs pull (case, cell tile, velocity chunk)
//                items from an atomic queue ordered by decreasing cost; each
//                thread owns cells of the tile and sweeps the chunk's
//                velocities (the kinetic pass of dvm_kinetic.cu with per-case
//                geometry), writing its chunk's partial moment sums.
//   k_b_finalize all cells of all cases: the chunks' sums added in order,
//                U^{n+1}, nu, mu and next parameters.
// The launch (threads per CTA, cells per thread, velocity chunks, CTAs per
// SM) is chosen by dvm_batch_autotune.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "dvm_internal.cuh"
#include "dvm_math.cuh"
#include "dvm_readback.cuh"

namespace dvm {
namespace {

// One case.  1D: nx cells, nv velocities from kmin, boundary rule bc.  2D
// (periodic in both dimensions): nx x ny cells (x fastest), nv x nvy
// velocities from (kmin, kminy).
struct BCase {
  int d;
  int nx, ny, nv, nvy, kmin, kminy, p, bc, forced_sub;
  int ghost_off, all_free;
  int ncell, nvel;   // cells and velocities of the case
  int nch;           // velocity chunks of its kinetic items
  long long f_off, c_off, e_off;  // pieces, cells, Euler state (2D, TW elements)
  double dx, dv, dt, w;
  double A[16];      // (C C^T)^{-1}, (d + 2)^2
  float Af[16];      // the same in FP32 (end-of-step arithmetic of FP32 builds)
};

struct BItem {
  int bcase, x0, chunk;
};

struct BPtrs {
  const BCase* cases;
  int ncases;
  const int* cell_case;
  long long ncells;
  const BItem* items;
  int nitems;
  void* F;
  void* ghost;
  double *U, *lam, *UE, *UM, *Us;  // nmb x ncells
  double* acc;       // [chunk][2 nmb][ncells] partial moment sums
  void* escr;        // Euler state of the 2D cases (W0, W1, split fluxes)
  int nmb;           // moment rows of the batch: 2 + the largest dimension
  void* prm;
  double* eqp;
  int* msub;
  double* alpha;
  int* status;
  long long* step;
  unsigned* qcounter;
  const int* order;   // cases by decreasing Euler cost (largest first)
  const int* order2;  // the 2D cases, by decreasing Euler cost
  int scheme;
  int cpt;  // cells per kinetic thread
};

constexpr int kB = 256;
// threads of a batched Euler CTA (one tube): the tube's cells per thread, and
// so the sub-step latency of the largest tubes, fall as it grows
#ifndef DVM_BATCH_EULER_THREADS
#define DVM_BATCH_EULER_THREADS 512
#endif
constexpr int kBE = DVM_BATCH_EULER_THREADS;
constexpr int kMaxBatchNx = 4096;      // 1D tube length (shared-memory Euler)
constexpr int kMaxBatchCells2D = 1 << 20;
constexpr int kMaxChunks = 4;          // velocity chunks of a case
// unrolling of the 1D tubes' velocity loop (loads of several velocities in
// flight; DVM_BATCH_UNROLL overrides it in launch-shape sweeps)
#ifndef DVM_BATCH_UNROLL
#define DVM_BATCH_UNROLL 2
#endif
constexpr int kBatchUnroll = DVM_BATCH_UNROLL;

// mu of Eq. minimMax for one cell of a 1D case (separable sums: one axis).
__device__ int b_cell_mu(const BCase& bc, const double* Uc, double mu[3], double& rho, double& u,
                         double& theta) {
  for (int i = 0; i < 3; ++i)
    if (!isfinite(Uc[i])) return DVM_ERR_NONFINITE;
  double uu[3];
  primitives<1>(Uc, rho, uu, theta);
  u = uu[0];
  if (!(rho > 0.0) || !(theta > 0.0)) return DVM_ERR_NONPHYSICAL;
  double G0, G1, G2;
  gauss_axis_sums(bc.nv, bc.kmin, bc.dv, u, theta, G0, G1, G2);
  const double pref = bc.w * rho / sqrt(2.0 * M_PI * theta);
  const double CM[3] = {pref * G0, pref * G1, 0.5 * pref * G2};
  double r[3];
  for (int i = 0; i < 3; ++i) r[i] = Uc[i] - CM[i];
  for (int i = 0; i < 3; ++i) mu[i] = bc.A[3 * i] * r[0] + bc.A[3 * i + 1] * r[1] + bc.A[3 * i + 2] * r[2];
  return 0;
}

// Per-cell parameters in the grouped layout of dvm_internal.cuh.
template <int D, typename TC>
__device__ void b_write_params(const BCase& bc, TC* prm, long long c, long long nc, double lam,
                               double weight, double rho, const double* u, double theta, const double* nu,
                               const double* mu) {
  TC L, h;
  if (sizeof(TC) == 8) {
    L = (TC)(log2(weight) + log2(rho) - 0.5 * D * log2(2.0 * M_PI * theta));
    h = (TC)(M_LOG2E * 0.5 / theta);
  } else {
    L = (TC)(log2f((float)weight) + log2f((float)rho) -
             0.5f * D * log2f(6.283185307179586f * (float)theta));
    h = (TC)(0.72134752044448170f / (float)theta);
  }
  prm[prm_at(row_lam(), c, nc)] = (TC)lam;
  prm[prm_at(row_L(), c, nc)] = L;
  for (int i = 0; i < D; ++i) prm[prm_at(row_u(i), c, nc)] = (TC)u[i];
  prm[prm_at(row_h(D), c, nc)] = h;
  for (int i = 0; i < D + 2; ++i) {
    const double e = i == D + 1 ? 0.5 : 1.0;  // energy row: coefficient of |v|^2
    prm[prm_at(row_nu(D, i), c, nc)] = (TC)(nu ? e * bc.w * nu[i] : 0.0);
    prm[prm_at(row_mu(D, i), c, nc)] = (TC)(e * weight * bc.w * mu[i]);
  }
}

// The velocity set of a 2D case in the form the single-problem helpers read
// (cell_mu: velocity counts, first indices, spacing and weight).
__device__ inline Geom b_geom2(const BCase& bc) {
  Geom g;
  g.d = 2;
  g.nm = 4;
  g.nv[0] = bc.nv;
  g.nv[1] = bc.nvy;
  g.nv[2] = 1;
  g.kmin[0] = bc.kmin;
  g.kmin[1] = bc.kminy;
  g.kmin[2] = 0;
  g.dv = bc.dv;
  g.w = bc.w;
  return g;
}

// mu and the primitive variables of one cell of case bc (1D or 2D).
__device__ int b_any_mu(const BCase& bc, const double* A, const double* Uc, double* mu, double& rho,
                        double u[3], double& theta) {
  if (bc.d == 1) {
    u[1] = u[2] = 0.0;
    return b_cell_mu(bc, Uc, mu, rho, u[0], theta);
  }
  const Geom g = b_geom2(bc);
  return cell_mu<2>(g, A, Uc, mu, rho, u, theta);
}

// FP32-storage builds: primitives, the Gaussian sums and mu = A (U - C M[U])
// in FP32, C M[U] and U - C M[U] in FP64 (as cell_mu_f32 for one problem).
__device__ int b_cell_mu_f32(const BCase& bc, const double* Uc, float mu[3], float& rho, float& u,
                             float& theta) {
  for (int i = 0; i < 3; ++i)
    if (!isfinite(Uc[i])) return DVM_ERR_NONFINITE;
  if (!(Uc[0] > 0.0)) return DVM_ERR_NONPHYSICAL;
  rho = (float)Uc[0];
  const float ir = 1.f / rho;
  u = (float)Uc[1] * ir;
  theta = 2.f * (float)Uc[2] * ir - u * u;
  if (!(theta > 0.f) || !(rho > 0.f)) {
    double rd, ud[3], td;
    primitives<1>(Uc, rd, ud, td);
    if (!(rd > 0.0) || !(td > 0.0)) return DVM_ERR_NONPHYSICAL;
    rho = (float)rd, u = (float)ud[0], theta = (float)td;
    if (!(theta > 0.f) || !(rho > 0.f)) return DVM_ERR_NONPHYSICAL;
  }
  double G0, G1, G2;
  gauss_axis_sums_f32(bc.nv, bc.kmin, (float)bc.dv, u, theta, G0, G1, G2);
  const double pref = bc.w * (double)rho * (double)rsqrtf(6.283185307179586f * theta);
  const double CM[3] = {pref * G0, pref * G1, 0.5 * pref * G2};
  float r[3];
  for (int i = 0; i < 3; ++i) r[i] = (float)(Uc[i] - CM[i]);
  for (int i = 0; i < 3; ++i) mu[i] = fmaf(bc.Af[3 * i], r[0], fmaf(bc.Af[3 * i + 1], r[1], bc.Af[3 * i + 2] * r[2]));
  return 0;
}

__device__ int b_any_mu_f32(const BCase& bc, const double* Uc, float* mu, float& rho, float u[3],
                            float& theta) {
  if (bc.d == 1) {
    u[1] = u[2] = 0.f;
    return b_cell_mu_f32(bc, Uc, mu, rho, u[0], theta);
  }
  const Geom g = b_geom2(bc);
  return cell_mu_f32<2>(g, bc.Af, Uc, mu, rho, u, theta);
}

template <int D>
__device__ void b_write_params_f32(const BCase& bc, float* prm, long long c, long long nc, float lam,
                                   float weight, float rho, const float* u, float theta, const float* nu,
                                   const float* mu) {
  prm[prm_at(row_lam(), c, nc)] = lam;
  prm[prm_at(row_L(), c, nc)] = log2f(weight) + log2f(rho) - 0.5f * D * log2f(6.283185307179586f * theta);
  for (int i = 0; i < D; ++i) prm[prm_at(row_u(i), c, nc)] = u[i];
  prm[prm_at(row_h(D), c, nc)] = 0.72134752044448170f / theta;
  const float w = (float)bc.w;
  for (int i = 0; i < D + 2; ++i) {
    const float e = i == D + 1 ? 0.5f : 1.f;  // energy row: coefficient of |v|^2
    prm[prm_at(row_nu(D, i), c, nc)] = nu ? e * w * nu[i] : 0.f;
    prm[prm_at(row_mu(D, i), c, nc)] = e * weight * w * mu[i];
  }
}

template <typename TC>
__global__ void k_b_cell_params(BPtrs p, int mode, int initial) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= p.ncells) return;
  const BCase& bc = p.cases[p.cell_case[c]];
  const int nm = bc.d + 2;
  double Uc[4], mu[4], rho, u[3], theta;
  for (int i = 0; i < nm; ++i) Uc[i] = p.U[i * p.ncells + c];
  const double lam = p.lam[c];
  if (mode == 0) {
    const int rc = b_any_mu(bc, bc.A, Uc, mu, rho, u, theta);
    if (rc) { set_status(p.status, rc); return; }
    if (bc.d == 1) b_write_params<1, double>(bc, p.eqp, c, p.ncells, lam, 1.0, rho, u, theta, nullptr, mu);
    else b_write_params<2, double>(bc, p.eqp, c, p.ncells, lam, 1.0, rho, u, theta, nullptr, mu);
    return;
  }
  const double weight = (p.scheme == DVM_FKS && initial) ? 0.0 : 1.0 - lam;
  if constexpr (sizeof(TC) == 4) {
    float muf[4], rf, uf[3], tf;
    const int rc = b_any_mu_f32(bc, Uc, muf, rf, uf, tf);
    if (rc) { set_status(p.status, rc); return; }
    if (bc.d == 1) b_write_params_f32<1>(bc, (float*)p.prm, c, p.ncells, (float)lam, (float)weight, rf, uf, tf, nullptr, muf);
    else b_write_params_f32<2>(bc, (float*)p.prm, c, p.ncells, (float)lam, (float)weight, rf, uf, tf, nullptr, muf);
  } else {
    const int rc = b_any_mu(bc, bc.A, Uc, mu, rho, u, theta);
    if (rc) { set_status(p.status, rc); return; }
    if (bc.d == 1) b_write_params<1, TC>(bc, (TC*)p.prm, c, p.ncells, lam, weight, rho, u, theta, nullptr, mu);
    else b_write_params<2, TC>(bc, (TC*)p.prm, c, p.ncells, lam, weight, rho, u, theta, nullptr, mu);
  }
}

// f^0 = E[U^0] for the points of one case (grid: chunks x cases).
template <typename TS, typename TC>
__global__ void k_b_init_f(BPtrs p) {
  const BCase& bc = p.cases[blockIdx.y];
  const long long npts = (long long)bc.ncell * bc.nvel;
  const long long nc = p.ncells;
  const double* e = p.eqp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / bc.ncell), cl = (int)(i % bc.ncell);
    const long long c = bc.c_off + cl;
    TC f;
    if (bc.d == 1) {
      const TC v = (TC)((double)(bc.kmin + k) * bc.dv);
      const TC du = v - (TC)e[prm_at(row_u(0), c, nc)];
      const TC lin = (TC)e[prm_at(row_mu(1, 0), c, nc)] + (TC)e[prm_at(row_mu(1, 1), c, nc)] * v +
                     (TC)e[prm_at(row_mu(1, 2), c, nc)] * v * v;
      const TC ex = (TC)e[prm_at(row_L(), c, nc)] - (TC)e[prm_at(row_h(1), c, nc)] * du * du;
      f = (sizeof(TC) == 8 ? (TC)exp2((double)ex) : (TC)exp2f((float)ex)) + lin;
    } else {
      const TC vx = (TC)((double)(bc.kmin + k % bc.nv) * bc.dv);
      const TC vy = (TC)((double)(bc.kminy + k / bc.nv) * bc.dv);
      const TC dx = vx - (TC)e[prm_at(row_u(0), c, nc)], dy = vy - (TC)e[prm_at(row_u(1), c, nc)];
      const TC lin = (TC)e[prm_at(row_mu(2, 0), c, nc)] + (TC)e[prm_at(row_mu(2, 1), c, nc)] * vx +
                     (TC)e[prm_at(row_mu(2, 2), c, nc)] * vy +
                     (TC)e[prm_at(row_mu(2, 3), c, nc)] * (vx * vx + vy * vy);
      const TC ex = (TC)e[prm_at(row_L(), c, nc)] - (TC)e[prm_at(row_h(2), c, nc)] * (dx * dx + dy * dy);
      f = (sizeof(TC) == 8 ? (TC)exp2((double)ex) : (TC)exp2f((float)ex)) + lin;
    }
    StoreT<TS>::store((TS*)p.F + bc.f_off + i, f);
  }
}

__device__ inline int b_index(int t, int n, int bc) {
  if (bc == DVM_BC_PERIODIC) {
    if (t >= 0 && t < n) return t;
    const int r = t % n;
    return r < 0 ? r + n : r;
  }
  return t < 0 ? 0 : (t >= n ? n - 1 : t);
}

// One CTA per case: alpha, m, MUSCL sub-steps in shared memory, U_E; outflow
// boundary pieces; queue reset.
// Start of a step, one CTA per case: the outflow cases' boundary pieces of
// every velocity at time n (read by the kinetic pass for sources outside the
// tube) and the reset of the kinetic work queue.
template <typename TS>
__global__ void k_b_prepare(BPtrs p) {
  const int ci = blockIdx.x, tid = threadIdx.x;
  const BCase& bc = p.cases[ci];
  const int nx = bc.nx;
  if (ci == 0 && tid == 0) *p.qcounter = 0u;
  if (bc.bc != DVM_BC_OUTFLOW) return;
  const long long n = *p.step;
  const TS* F = (const TS*)p.F + bc.f_off;
  TS* G = (TS*)p.ghost + bc.ghost_off;
  for (int k = tid; k < bc.nv; k += blockDim.x) {
    const long long o = transport_offset(bc.kmin + k, n, bc.p);
    G[2 * k] = F[(long long)k * nx + wrap(0 - o, nx)];
    G[2 * k + 1] = F[(long long)k * nx + wrap((long long)(nx - 1) - o, nx)];
  }
}

// All MUSCL sub-steps of one 2D case by one CTA (Section 4.3.2 with the
// unsplit sum of the x and y flux differences): the state W and the split
// fluxes G+- = F +- alpha_i W of both directions live in global memory (the
// case's slice of p.escr, L2-resident); alpha per direction of every
// sub-step's initial state, sub-step length dx / (2 (alpha_x + alpha_y)) of
// Eq. Time2, the last one ending at dt.
template <typename TW, bool LIMITED>
__device__ void b_euler_2d(const BPtrs& p, const BCase& bc, int ci) {
  __shared__ TW s_red2[2][kBE / 32];
  __shared__ double s_dt2;
  __shared__ TW s_kk2, s_ax, s_ay;
  __shared__ int s_fl2;
  const int tid = threadIdx.x;
  const int nx = bc.nx, ny = bc.ny, ncl = bc.ncell;
  const long long nc = p.ncells;
  TW* W0 = (TW*)p.escr + bc.e_off;
  TW* W1 = W0 + 4 * (size_t)ncl;
  TW* G = W1 + 4 * (size_t)ncl;  // [dir][+/-][component][cell]
  TW ax = TW(0), ay = TW(0);
  for (int c = tid; c < ncl; c += kBE) {
    const double w = bc.all_free ? 0.0 : 1.0 - p.lam[bc.c_off + c];
    TW W[4];
    for (int i = 0; i < 4; ++i) {
      W[i] = (TW)(w * p.U[i * nc + bc.c_off + c]);
      W0[i * ncl + c] = W[i];
    }
    TW a[3];
    state_alpha_of<2>(W, a);
    ax = ax > a[0] ? ax : a[0];
    ay = ay > a[1] ? ay : a[1];
  }
  double t = 0.0, a0x = 0.0, a0y = 0.0;
  int s = 0;
  for (;; ++s) {
    for (int o = 16; o > 0; o >>= 1) {
      const TW vx = __shfl_xor_sync(0xffffffffu, ax, o), vy = __shfl_xor_sync(0xffffffffu, ay, o);
      ax = ax > vx ? ax : vx;
      ay = ay > vy ? ay : vy;
    }
    if ((tid & 31) == 0) {
      s_red2[0][tid >> 5] = ax;
      s_red2[1][tid >> 5] = ay;
    }
    __syncthreads();
    if (tid == 0) {
      TW mx = TW(0), my = TW(0);
      for (int w = 0; w < kBE / 32; ++w) {
        mx = mx > s_red2[0][w] ? mx : s_red2[0][w];
        my = my > s_red2[1][w] ? my : s_red2[1][w];
      }
      if (s == 0) a0x = (double)mx, a0y = (double)my;
      int flags = 0;
      double dtE = 0.0;
      const double asum = sizeof(TW) == 8 ? __dadd_rn((double)mx, (double)my) : (double)(mx + my);
      if (bc.all_free) {
        flags = 2;
      } else if (bc.forced_sub > 0) {
        dtE = bc.dt / bc.forced_sub;
        flags = (s + 1 == bc.forced_sub) ? 1 : 0;
      } else if (!(asum > 0.0)) {
        set_status(p.status, DVM_ERR_NONPHYSICAL);
        flags = 2;
      } else {
        const double cfl = sizeof(TW) == 8 ? __ddiv_rn(__dmul_rn(0.5, bc.dx), asum)
                                           : (double)__fdiv_rn(0.5f * (float)bc.dx, (float)asum);
        const double rem = __dsub_rn(bc.dt, t);
        flags = cfl >= rem ? 1 : 0;
        dtE = flags ? rem : cfl;
      }
      s_dt2 = dtE;
      s_kk2 = sizeof(TW) == 8 ? (TW)(dtE / bc.dx) : (TW)((float)dtE / (float)bc.dx);
      s_ax = mx;
      s_ay = my;
      s_fl2 = flags;
      t = __dadd_rn(t, dtE);
    }
    __syncthreads();
    const int flags = s_fl2;
    if (flags & 2) break;
    const bool last = (flags & 1) != 0;
    const TW kk = s_kk2, alx = s_ax, aly = s_ay;
    const TW* src = (s & 1) ? W1 : W0;
    TW* dst = (s & 1) ? W0 : W1;
    // split fluxes of every cell in both directions
    for (int c = tid; c < ncl; c += kBE) {
      TW U[4], Fx[4], Fy[4];
      for (int i = 0; i < 4; ++i) U[i] = src[i * ncl + c];
      euler_flux<TW, 2>(U, 0, Fx);
      euler_flux<TW, 2>(U, 1, Fy);
      for (int i = 0; i < 4; ++i) {
        G[(0 * 4 + i) * ncl + c] = Fx[i] + alx * U[i];
        G[(1 * 4 + i) * ncl + c] = Fx[i] - alx * U[i];
        G[(2 * 4 + i) * ncl + c] = Fy[i] + aly * U[i];
        G[(3 * 4 + i) * ncl + c] = Fy[i] - aly * U[i];
      }
    }
    __syncthreads();
    ax = ay = TW(0);
    for (int c = tid; c < ncl; c += kBE) {
      const int x = c % nx, y = c / nx;
      int sx[5], sy[5];  // the stencil cells -2 .. +2 along x and y (periodic)
      for (int o = 0; o < 5; ++o) {
        sx[o] = y * nx + b_index(x + o - 2, nx, DVM_BC_PERIODIC);
        sy[o] = b_index(y + o - 2, ny, DVM_BC_PERIODIC) * nx + x;
      }
      TW Wn[4];
      for (int i = 0; i < 4; ++i) {
        TW dif = TW(0);
        for (int dir = 0; dir < 2; ++dir) {
          const int* st = dir == 0 ? sx : sy;
          const TW* gp = G + ((2 * dir) * 4 + i) * (size_t)ncl;
          const TW* gm = G + ((2 * dir + 1) * 4 + i) * (size_t)ncl;
          TW psi[2];
          for (int f = 0; f < 2; ++f) {
            const int j = 1 + f;  // face between stencil cells j and j + 1
            const TW sp = slope<TW, LIMITED>(gp[st[j]] - gp[st[j - 1]], gp[st[j + 1]] - gp[st[j]]);
            const TW sm = slope<TW, LIMITED>(gm[st[j + 1]] - gm[st[j]], gm[st[j + 2]] - gm[st[j + 1]]);
            psi[f] = TW(0.5) * (gp[st[j]] + gm[st[j + 1]]) + TW(0.25) * (sp - sm);
          }
          dif += psi[1] - psi[0];
        }
        Wn[i] = src[i * ncl + c] - kk * dif;
        dst[i * ncl + c] = Wn[i];
      }
      if (!last) {
        TW a[3];
        state_alpha_of<2>(Wn, a);
        ax = ax > a[0] ? ax : a[0];
        ay = ay > a[1] ? ay : a[1];
      }
    }
    __syncthreads();
    if (last) break;
    if (s + 1 >= 1000000) {
      if (tid == 0) set_status(p.status, DVM_ERR_CFL);
      break;
    }
  }
  const int m = bc.all_free ? 0 : s + 1;
  if (tid == 0) {
    p.msub[ci] = m;
    p.alpha[ci] = a0x + a0y;
  }
  const TW* res = (m & 1) ? W1 : W0;
  for (int c = tid; c < ncl; c += kBE)
    for (int i = 0; i < 4; ++i) p.UE[i * nc + bc.c_off + c] = (double)res[i * ncl + c];
}

// The 2D cases' Euler sub-steps (a launch of its own, so that the 1D kernel
// keeps its registers): CTA i takes 2D case order2[i].
template <typename TW, bool LIMITED>
__global__ void __launch_bounds__(kBE) k_b_euler2d(BPtrs p) {
  const int ci = p.order2[blockIdx.x];
  b_euler_2d<TW, LIMITED>(p, p.cases[ci], ci);
}

// All MUSCL sub-steps of one 1D case (CTA blockIdx.x takes case
// order[blockIdx.x]; 2D cases leave at once).
template <typename TS, typename TW, bool LIMITED, bool EULER, bool SPLIT>
__global__ void __launch_bounds__(kBE) k_b_euler(BPtrs p) {
  extern __shared__ unsigned char s_raw[];
  const int ci = p.order[blockIdx.x], tid = threadIdx.x;
  const BCase& bc = p.cases[ci];
  const int nx = bc.nx;
  const long long nc = p.ncells;
  if (!EULER || bc.d != 1) return;
  TW* W0 = reinterpret_cast<TW*>(s_raw);
  TW* W1 = W0 + 3 * nx;
  // W = (1 - lambda) U and the alpha of every sub-step's initial state (Eq.
  // Time2 per sub-step, the last one ending at dt).  alpha is reduced in the
  // state's type; the sub-step scalars are computed once per CTA by thread 0
  // (FP64 in the FP64 build, the quotient in FP32 otherwise) and broadcast.
  __shared__ TW s_redw[kBE / 32];
  __shared__ double s_dtE;
  __shared__ TW s_kk, s_alw;
  __shared__ int s_flags;  // bit 0: last sub-step, bit 1: stop (error or all free)
  TW amax = TW(0);
  for (int x = tid; x < nx; x += kBE) {
    const long long c = bc.c_off + x;
    const double w = bc.all_free ? 0.0 : 1.0 - p.lam[c];
    TW W[3];
    for (int i = 0; i < 3; ++i) {
      W[i] = (TW)(w * p.U[i * nc + c]);
      W0[i * nx + x] = W[i];
    }
    TW a[3];
    state_alpha_of<1>(W, a);
    amax = amax > a[0] ? amax : a[0];
  }
  double t = 0.0, a0 = 0.0;
  int s = 0;
  for (;; ++s) {
    for (int o = 16; o > 0; o >>= 1) {
      const TW v = __shfl_xor_sync(0xffffffffu, amax, o);
      amax = amax > v ? amax : v;
    }
    if ((tid & 31) == 0) s_redw[tid >> 5] = amax;
    __syncthreads();
    if (tid == 0) {
      TW alt = TW(0);
      for (int w = 0; w < kBE / 32; ++w) alt = alt > s_redw[w] ? alt : s_redw[w];
      const double al = (double)alt;
      if (s == 0) a0 = al;
      int flags = 0;
      double dtE = 0.0;
      if (bc.all_free) {
        flags = 2;
      } else if (bc.forced_sub > 0) {
        dtE = bc.dt / bc.forced_sub;
        flags = (s + 1 == bc.forced_sub) ? 1 : 0;
      } else if (!(al > 0.0)) {
        set_status(p.status, DVM_ERR_NONPHYSICAL);
        flags = 2;
      } else {
        const double cfl = sizeof(TW) == 8 ? __ddiv_rn(__dmul_rn(0.5, bc.dx), al)
                                           : (double)__fdiv_rn(0.5f * (float)bc.dx, (float)al);
        const double rem = __dsub_rn(bc.dt, t);
        flags = cfl >= rem ? 1 : 0;
        dtE = flags ? rem : cfl;
      }
      s_dtE = dtE;
      s_kk = sizeof(TW) == 8 ? (TW)(dtE / bc.dx) : (TW)((float)dtE / (float)bc.dx);
      s_alw = alt;
      s_flags = flags;
      t = __dadd_rn(t, dtE);
    }
    __syncthreads();
    const int flags = s_flags;
    if (flags & 2) break;
    const bool last = (flags & 1) != 0;
    const TW kk = s_kk, alw = s_alw;
    const TW* src = (s & 1) ? W1 : W0;
    TW* dst = (s & 1) ? W0 : W1;
    amax = TW(0);
    if (SPLIT) {
      // split fluxes G+- = F +- alpha W once per cell, then the two faces of
      // every cell from them (boundary cells by the case's rule)
      TW* Gp = W1 + 3 * nx;
      TW* Gm = Gp + 3 * nx;
      for (int x = tid; x < nx; x += kBE) {
        TW U[3], F[3];
        for (int i = 0; i < 3; ++i) U[i] = src[i * nx + x];
        euler_flux<TW, 1>(U, 0, F);
        for (int i = 0; i < 3; ++i) {
          Gp[i * nx + x] = F[i] + alw * U[i];
          Gm[i * nx + x] = F[i] - alw * U[i];
        }
      }
      __syncthreads();
      for (int x = tid; x < nx; x += kBE) {
        int xx[5];
        for (int o = 0; o < 5; ++o) xx[o] = b_index(x + o - 2, nx, bc.bc);
        TW Wn[3];
        for (int i = 0; i < 3; ++i) {
          const TW* gp = Gp + i * nx;
          const TW* gm = Gm + i * nx;
          TW psi[2];
          for (int f = 0; f < 2; ++f) {
            const int j = 1 + f;  // face between cells j and j + 1 of the stencil
            const TW sp = slope<TW, LIMITED>(gp[xx[j]] - gp[xx[j - 1]], gp[xx[j + 1]] - gp[xx[j]]);
            const TW sm = slope<TW, LIMITED>(gm[xx[j + 1]] - gm[xx[j]], gm[xx[j + 2]] - gm[xx[j + 1]]);
            psi[f] = TW(0.5) * (gp[xx[j]] + gm[xx[j + 1]]) + TW(0.25) * (sp - sm);
          }
          Wn[i] = src[i * nx + x] - kk * (psi[1] - psi[0]);
          dst[i * nx + x] = Wn[i];
        }
        if (!last) {
          TW a[3];
          state_alpha_of<1>(Wn, a);
          amax = amax > a[0] ? amax : a[0];
        }
      }
    } else {
    for (int x = tid; x < nx; x += kBE) {
      TW Us[5][3], Fs[5][3], Wn[3];
      for (int o = 0; o < 5; ++o) {
        const int xx = b_index(x + o - 2, nx, bc.bc);
        for (int i = 0; i < 3; ++i) Us[o][i] = src[i * nx + xx];
        euler_flux<TW, 1>(Us[o], 0, Fs[o]);
      }
      for (int i = 0; i < 3; ++i) {
        TW Gp[5], Gm[5], psi[2];
        for (int o = 0; o < 5; ++o) {
          Gp[o] = Fs[o][i] + alw * Us[o][i];
          Gm[o] = Fs[o][i] - alw * Us[o][i];
        }
        for (int f = 0; f < 2; ++f) {
          const int j = 1 + f;
          const TW sp = slope<TW, LIMITED>(Gp[j] - Gp[j - 1], Gp[j + 1] - Gp[j]);
          const TW sm = slope<TW, LIMITED>(Gm[j + 1] - Gm[j], Gm[j + 2] - Gm[j + 1]);
          psi[f] = TW(0.5) * (Fs[j][i] + Fs[j + 1][i]) - TW(0.5) * alw * (Us[j + 1][i] - Us[j][i]) +
                   TW(0.25) * (sp - sm);
        }
        Wn[i] = Us[2][i] - kk * (psi[1] - psi[0]);
        dst[i * nx + x] = Wn[i];
      }
      if (!last) {
        TW a[3];
        state_alpha_of<1>(Wn, a);
        amax = amax > a[0] ? amax : a[0];
      }
    }
    }
    __syncthreads();
    if (last) break;
    if (s + 1 >= 1000000) {
      if (tid == 0) set_status(p.status, DVM_ERR_CFL);
      break;
    }
  }
  const int m = bc.all_free ? 0 : s + 1;
  if (tid == 0) {
    p.msub[ci] = m;
    p.alpha[ci] = a0;
  }
  const TW* res = (m & 1) ? W1 : W0;
  for (int x = tid; x < nx; x += kBE)
    for (int i = 0; i < 3; ++i) p.UE[i * nc + bc.c_off + x] = (double)res[i * nx + x];
}

// Kinetic pass of one cell tile and velocity chunk of a 2D case (periodic):
// the generic pass of dvm_kinetic.cu with the case's geometry; FP32 sums per
// velocity row, FP64 across rows, this chunk's partial sums written to its
// slice of p.acc.
template <typename TS, typename TC, bool HOFKS>
__device__ void b_kinetic_2d(const BPtrs& p, const BCase& bc, const BItem& item, long long n,
                             int (*s_slot)[kMaxV1], int (*s_delta)[kMaxV1], TC (*s_v)[kMaxV1]) {
  const long long nc = p.ncells;
  const TC* prm = (const TC*)p.prm;
  TS* F = (TS*)p.F + bc.f_off;
  const int nx = bc.nx, ny = bc.ny, ncl = bc.ncell;
  const int kb = (int)((long long)item.chunk * bc.nvel / bc.nch);
  const int ke = (int)((long long)(item.chunk + 1) * bc.nvel / bc.nch);
  for (int j = 0; j < p.cpt; ++j) {
    const int cl = item.x0 + threadIdx.x + j * blockDim.x;
    if (cl >= ncl) break;
    const int x = cl % nx, y = cl / nx;
    const long long c = bc.c_off + cl;
    const TC lam_c = prm[prm_at(row_lam(), c, nc)];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    TC r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int kx = kb % bc.nv, ky = kb / bc.nv;
    for (int k = kb; k < ke; ++k) {
      int sx = x - s_delta[0][kx], sy = y - s_delta[1][ky];
      sx = b_index(sx, nx, DVM_BC_PERIODIC);
      sy = b_index(sy, ny, DVM_BC_PERIODIC);
      int qx = x - s_slot[0][kx], qy = y - s_slot[1][ky];
      if (qx < 0) qx += nx;
      if (qy < 0) qy += ny;
      const TC fv = StoreT<TS>::load(F + (long long)k * ncl + qy * nx + qx);
      const long long cs = bc.c_off + sy * nx + sx;
      const TC vx = s_v[0][kx], vy = s_v[1][ky];
      const TC v2 = vx * vx + vy * vy;
      // source parameters (d = 2 rows: lambda L ux uy | h nu0 nu1 nu2 | nu3 mu0 mu1 mu2 | mu3)
      TC plam, pL, pux, puy, ph, n0, n1, n2, n3, m0, m1, m2, m3;
      if constexpr (sizeof(TC) == 4) {
        const float4* pg = reinterpret_cast<const float4*>(prm);
        const float4 g0 = __ldg(pg + cs), g1 = __ldg(pg + nc + cs), g2 = __ldg(pg + 2 * nc + cs),
                     g3 = __ldg(pg + 3 * nc + cs);
        plam = g0.x; pL = g0.y; pux = g0.z; puy = g0.w;
        ph = g1.x; n0 = g1.y; n1 = g1.z; n2 = g1.w;
        n3 = g2.x; m0 = g2.y; m1 = g2.z; m2 = g2.w;
        m3 = g3.x;
      } else {
        plam = prm[prm_at(row_lam(), cs, nc)];
        pL = prm[prm_at(row_L(), cs, nc)];
        pux = prm[prm_at(row_u(0), cs, nc)];
        puy = prm[prm_at(row_u(1), cs, nc)];
        ph = prm[prm_at(row_h(2), cs, nc)];
        n0 = prm[prm_at(row_nu(2, 0), cs, nc)];
        n1 = prm[prm_at(row_nu(2, 1), cs, nc)];
        n2 = prm[prm_at(row_nu(2, 2), cs, nc)];
        n3 = prm[prm_at(row_nu(2, 3), cs, nc)];
        m0 = prm[prm_at(row_mu(2, 0), cs, nc)];
        m1 = prm[prm_at(row_mu(2, 1), cs, nc)];
        m2 = prm[prm_at(row_mu(2, 2), cs, nc)];
        m3 = prm[prm_at(row_mu(2, 3), cs, nc)];
      }
      const TC dx = vx - pux, dy = vy - puy;
      const TC ex = pL - ph * (dx * dx + dy * dy);
      TC M;
      if constexpr (sizeof(TC) == 8) {
        M = (TC)exp2((double)ex);
      } else {
        float yv;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(yv) : "f"((float)ex));
        M = yv;
      }
      const TC lm = m0 + m1 * vx + m2 * vy + m3 * v2;
      TC fnew;
      if (HOFKS) {
        const TC ln = n0 + n1 * vx + n2 * vy + n3 * v2;
        const TC a = plam * (fv + ln);  // T(lambda f^n)
        const TC b = M + lm;            // T((1 - lambda) E^n)
        fnew = a + b;
        r[0] += a; r[1] += a * vx; r[2] += a * vy; r[3] += a * v2;
        r[4] += b; r[5] += b * vx; r[6] += b * vy; r[7] += b * v2;
      } else {
        const TC fs = fv + M + lm;
        fnew = lam_c * fs;
        r[0] += fs; r[1] += fs * vx; r[2] += fs * vy; r[3] += fs * v2;
      }
      StoreT<TS>::store(F + (long long)k * ncl + qy * nx + qx, fnew);
      if (++kx == bc.nv) {  // end of a velocity row: FP32 row sums into FP64
        kx = 0;
        ++ky;
        for (int t = 0; t < 8; ++t) acc[t] += (double)r[t], r[t] = TC(0);
      }
    }
    for (int t = 0; t < 8; ++t) acc[t] += (double)r[t];
    // rows of the chunk's slice: the a part at 0..3, the b part at nmb..nmb+3
    double* out = p.acc + (long long)item.chunk * 2 * p.nmb * nc + c;
    for (int t = 0; t < (HOFKS ? 8 : 4); ++t)
      out[(t / 4 * p.nmb + t % 4) * nc] = (t % 4 == 3 ? 0.5 : 1.0) * acc[t];
  }
}

// Persistent kinetic pass over (case, tile, velocity chunk) items (D2: the
// batch has 2D cases; without them their path is not compiled in).
template <typename TS, typename TC, bool HOFKS, bool D2>
__global__ void k_b_kinetic(BPtrs p) {
  __shared__ int s_item;
  __shared__ BCase s_case;
  __shared__ int s_slot[D2 ? 2 : 1][kMaxV1], s_delta[D2 ? 2 : 1][kMaxV1];
  __shared__ TC s_v[D2 ? 2 : 1][kMaxV1];
  const long long n = *p.step;
  const long long nc = p.ncells;
  const TC* prm = (const TC*)p.prm;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(p.qcounter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= p.nitems) return;
    const BItem item = p.items[it];
    if (threadIdx.x == 0) s_case = p.cases[item.bcase];
    __syncthreads();
    const BCase& bc = s_case;
    for (int t = threadIdx.x; t < (D2 ? 2 : 1) * kMaxV1; t += blockDim.x) {
      const int dim = t / kMaxV1, k = t % kMaxV1;
      if (k >= (dim == 0 ? bc.nv : (bc.d == 2 ? bc.nvy : 0))) continue;
      const long long kg = (dim == 0 ? bc.kmin : bc.kminy) + k;
      const int N = dim == 0 ? bc.nx : bc.ny;
      const long long o1 = transport_offset(kg, n + 1, bc.p);
      s_slot[dim][k] = wrap(o1, N);
      s_delta[dim][k] = (int)(o1 - transport_offset(kg, n, bc.p));
      s_v[dim][k] = (TC)((double)kg * bc.dv);
    }
    __syncthreads();
    if constexpr (D2) {
      if (bc.d == 2) {
        b_kinetic_2d<TS, TC, HOFKS>(p, bc, item, n, s_slot, s_delta, s_v);
        continue;
      }
    }
    const TS* G = (const TS*)p.ghost + bc.ghost_off;
    TS* F = (TS*)p.F + bc.f_off;
    const int kb = (int)((long long)item.chunk * bc.nv / bc.nch);
    const int ke = (int)((long long)(item.chunk + 1) * bc.nv / bc.nch);
    for (int j = 0; j < p.cpt; ++j) {
      const int x = item.x0 + threadIdx.x + j * blockDim.x;
      if (x >= bc.nx) break;
      const long long c = bc.c_off + x;
      const TC lam_c = prm[prm_at(row_lam(), c, nc)];
      double acc[6] = {0, 0, 0, 0, 0, 0};
      TC r[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll kBatchUnroll
      for (int k = kb; k < ke; ++k) {
        int s = x - s_delta[0][k];
        bool clamped = false;
        if (bc.bc == DVM_BC_PERIODIC) {
          s = b_index(s, bc.nx, DVM_BC_PERIODIC);
        } else if (s < 0 || s >= bc.nx) {
          s = s < 0 ? 0 : bc.nx - 1;
          clamped = true;
        }
        int q = x - s_slot[0][k];
        if (q < 0) q += bc.nx;
        const TC fv = clamped ? StoreT<TS>::load(G + 2 * k + (s == 0 ? 0 : 1))
                              : StoreT<TS>::load(F + (long long)k * bc.nx + q);
        const long long cs = bc.c_off + s;
        const TC v = s_v[0][k];
        const TC v2 = v * v;
        // source parameters (d = 1 rows: lambda L u h | nu0 nu1 nu2 mu0 | mu1 mu2)
        TC plam, pL, pu, ph, n0, n1, n2, m0, m1, m2;
        if constexpr (sizeof(TC) == 4) {
          const float4* pg = reinterpret_cast<const float4*>(prm);
          const float4 g0 = __ldg(pg + cs), g1 = __ldg(pg + nc + cs), g2 = __ldg(pg + 2 * nc + cs);
          plam = g0.x; pL = g0.y; pu = g0.z; ph = g0.w;
          n0 = g1.x; n1 = g1.y; n2 = g1.z; m0 = g1.w;
          m1 = g2.x; m2 = g2.y;
        } else {
          plam = prm[prm_at(row_lam(), cs, nc)];
          pL = prm[prm_at(row_L(), cs, nc)];
          pu = prm[prm_at(row_u(0), cs, nc)];
          ph = prm[prm_at(row_h(1), cs, nc)];
          n0 = prm[prm_at(row_nu(1, 0), cs, nc)];
          n1 = prm[prm_at(row_nu(1, 1), cs, nc)];
          n2 = prm[prm_at(row_nu(1, 2), cs, nc)];
          m0 = prm[prm_at(row_mu(1, 0), cs, nc)];
          m1 = prm[prm_at(row_mu(1, 1), cs, nc)];
          m2 = prm[prm_at(row_mu(1, 2), cs, nc)];
        }
        const TC du = v - pu;
        const TC ex = pL - ph * du * du;
        TC M;
        if constexpr (sizeof(TC) == 8) {
          M = (TC)exp2((double)ex);
        } else {
          float y;
          asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"((float)ex));
          M = y;
        }
        const TC lm = m0 + m1 * v + m2 * v2;
        TC fnew;
        if (HOFKS) {
          const TC ln = n0 + n1 * v + n2 * v2;
          const TC a = plam * (fv + ln);  // T(lambda f^n)
          const TC b = M + lm;                                        // T((1 - lambda) E^n)
          fnew = a + b;
          r[0] += a; r[1] += a * v; r[2] += a * v2;
          r[3] += b; r[4] += b * v; r[5] += b * v2;
        } else {
          const TC fs = fv + M + lm;
          fnew = lam_c * fs;
          r[0] += fs; r[1] += fs * v; r[2] += fs * v2;
        }
        StoreT<TS>::store(F + (long long)k * bc.nx + q, fnew);
        if ((k & 31) == 31) {
          for (int t = 0; t < 6; ++t) acc[t] += (double)r[t], r[t] = TC(0);
        }
      }
      for (int t = 0; t < 6; ++t) acc[t] += (double)r[t];
      // rows t of the chunk's slice: the a part at 0..2, the b part at nmb..nmb+2
      double* out = p.acc + (long long)item.chunk * 2 * p.nmb * nc + c;
      for (int t = 0; t < (HOFKS ? 6 : 3); ++t)
        out[(t / 3 * p.nmb + t % 3) * nc] = (t % 3 == 2 ? 0.5 : 1.0) * acc[t];
    }
  }
}

// End of step for every cell of every case: the velocity chunks' partial
// sums added in chunk order, U^{n+1} = U_* + U_E, nu (Eq. minim_full), mu and
// the next step's parameters.
template <typename TC, bool HOFKS>
__global__ void k_b_finalize(BPtrs p) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c == 0) *p.step += 1;
  if (c >= p.ncells) return;
  const long long nc = p.ncells;
  const BCase& bc = p.cases[p.cell_case[c]];
  const int nm = bc.d + 2, nmb = p.nmb;
  double sa[4] = {0, 0, 0, 0}, sb[4] = {0, 0, 0, 0};
  for (int ch = 0; ch < bc.nch; ++ch) {
    const double* a = p.acc + (long long)ch * 2 * nmb * nc + c;
    for (int i = 0; i < nm; ++i) {
      sa[i] += a[i * nc];
      if (HOFKS) sb[i] += a[(nmb + i) * nc];
    }
  }
  double Un[4], r[4] = {0.0, 0.0, 0.0, 0.0};
  if (HOFKS) {
    for (int i = 0; i < nm; ++i) {
      const double us = bc.w * sa[i], um = bc.w * sb[i];
      const double ue = p.UE[i * nc + c];
      r[i] = ue - um;
      Un[i] = us + ue;
      p.Us[i * nc + c] = us;
      p.UM[i * nc + c] = um;
    }
  } else {
    for (int i = 0; i < nm; ++i) {
      Un[i] = bc.w * sa[i];
      p.Us[i * nc + c] = Un[i];
    }
  }
  for (int i = 0; i < nm; ++i) p.U[i * nc + c] = Un[i];
  const double lam = p.lam[c];
  // nu = A (U_E - U_M); FP32-storage builds: nu, mu and the primitives in FP32
  // (GB300's FP64 rate bounds this kernel otherwise), the moments in FP64
  if constexpr (sizeof(TC) == 4) {
    float nu[4], mu[4], rho, u[3], theta;
    for (int i = 0; i < nm; ++i) {
      float t = 0.f;
      for (int j = 0; j < nm; ++j) t = fmaf(bc.Af[i * nm + j], (float)r[j], t);
      nu[i] = t;
    }
    const int rc = b_any_mu_f32(bc, Un, mu, rho, u, theta);
    if (rc) { set_status(p.status, rc); return; }
    if (bc.d == 1)
      b_write_params_f32<1>(bc, (float*)p.prm, c, nc, (float)lam, (float)(1.0 - lam), rho, u, theta, HOFKS ? nu : nullptr, mu);
    else
      b_write_params_f32<2>(bc, (float*)p.prm, c, nc, (float)lam, (float)(1.0 - lam), rho, u, theta, HOFKS ? nu : nullptr, mu);
  } else {
    double nu[4], mu[4], rho, u[3], theta;
    for (int i = 0; i < nm; ++i) {
      double t = 0.0;
      for (int j = 0; j < nm; ++j) t += bc.A[i * nm + j] * r[j];
      nu[i] = t;
    }
    const int rc = b_any_mu(bc, bc.A, Un, mu, rho, u, theta);
    if (rc) { set_status(p.status, rc); return; }
    if (bc.d == 1)
      b_write_params<1, TC>(bc, (TC*)p.prm, c, nc, lam, 1.0 - lam, rho, u, theta, HOFKS ? nu : nullptr, mu);
    else
      b_write_params<2, TC>(bc, (TC*)p.prm, c, nc, lam, 1.0 - lam, rho, u, theta, HOFKS ? nu : nullptr, mu);
  }
}

// f of one case at the cell centres (stored piece + deferred term), FP64.
template <typename TS, typename TC>
__global__ void k_b_materialize(BPtrs p, int ci, double* out) {
  const BCase& bc = p.cases[ci];
  const long long npts = (long long)bc.ncell * bc.nvel;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const int k = (int)(i / bc.ncell), cl = (int)(i % bc.ncell);
  const long long n = *p.step, nc = p.ncells, c = bc.c_off + cl;
  const TC* prm = (const TC*)p.prm;
  const int D = bc.d;
  const int kk[2] = {D == 1 ? k : k % bc.nv, D == 1 ? 0 : k / bc.nv};
  const int kmin[2] = {bc.kmin, bc.kminy};
  const int N[2] = {bc.nx, bc.ny};
  const int xy[2] = {cl % bc.nx, cl / bc.nx};
  int q[2] = {0, 0};
  double v[2] = {0.0, 0.0}, v2 = 0.0;
  for (int dim = 0; dim < D; ++dim) {
    q[dim] = wrap((long long)xy[dim] - transport_offset(kmin[dim] + kk[dim], n, bc.p), N[dim]);
    v[dim] = (double)(kmin[dim] + kk[dim]) * bc.dv;
    v2 += v[dim] * v[dim];
  }
  double f = (double)StoreT<TS>::load((const TS*)p.F + bc.f_off + (long long)k * bc.ncell + q[1] * bc.nx + q[0]);
  // the deferred term of the cell (rows of dimension D)
  const int R = D + 2;
  auto rowv = [&](int base) {
    double t = (double)prm[prm_at(base, c, nc)] + (double)prm[prm_at(base + R - 1, c, nc)] * v2;
    for (int dim = 0; dim < D; ++dim) t += (double)prm[prm_at(base + 1 + dim, c, nc)] * v[dim];
    return t;
  };
  if (p.scheme == DVM_FKS) {
    double du2 = 0.0;
    for (int dim = 0; dim < D; ++dim) {
      const double du = v[dim] - (double)prm[prm_at(row_u(dim), c, nc)];
      du2 += du * du;
    }
    f += exp2((double)prm[prm_at(row_L(), c, nc)] - (double)prm[prm_at(row_h(D), c, nc)] * du2) +
         rowv(row_mu(D, 0));
  } else {
    f += rowv(row_nu(D, 0));
  }
  out[i] = f;
}

}  // namespace
}  // namespace dvm

using namespace dvm;

struct dvm_batch {
  std::vector<BCase> cases;
  std::vector<int> nxs;
  int ncases = 0;
  long long ncells = 0, npoints = 0;
  int precision = DVM_F32, scheme = DVM_HOFKS;
  int threads = 128, cpt = 1;
  int vch = 1;          // velocity chunks per case (at most; >= 16 velocities each)
  int ctas_per_sm = 0;  // resident kinetic CTAs per SM (0: as many as fit)
  int nmb = 3;          // moment rows: 2 + the largest dimension
  int n1d = 0, n2d = 0; // cases of each dimension
  int blocks = 0;
  int max_nx = 0;       // longest 1D tube (shared-memory Euler)
  size_t euler_smem = 0;
  bool split_euler = false;
  BPtrs p{};
  std::vector<void*> allocs;
  cudaStream_t stream = nullptr, cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* pinned = nullptr;
  int status = 0;
  std::string err;
  bool state_set = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t side = nullptr;       // high-priority stream of the Euler kernel
  cudaEvent_t fork = nullptr, join = nullptr;
  dvm::ReadBack rb;                  // dvm_batch_moments_async / _wait
};

namespace {

int bfail(dvm_batch* b, int code, const std::string& m) {
  if (b && b->status == 0) b->status = code;
  if (b) b->err = m;
  return code;
}

int bcheck(dvm_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return 0;
  return bfail(b, DVM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
int balloc(dvm_batch* b, T** ptr, size_t bytes) {
  void* q = nullptr;
  if (cudaMalloc(&q, bytes < 256 ? 256 : bytes) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, DVM_ERR_OOM, "batch allocation failed");
  }
  b->allocs.push_back(q);
  *ptr = (T*)q;
  return 0;
}

// Work items: tiles of threads * cpt cells times the case's velocity chunks,
// ordered by decreasing cost; the cases (with their chunk counts) uploaded.
int build_items(dvm_batch* b) {
  std::vector<std::pair<long long, BItem>> v;
  const int T = b->threads * b->cpt;
  for (int i = 0; i < b->ncases; ++i) {
    BCase& bc = b->cases[i];
    bc.nch = std::max(1, std::min(b->vch, bc.nvel / 16));
    for (int x0 = 0; x0 < bc.ncell; x0 += T)
      for (int ch = 0; ch < bc.nch; ++ch) {
        const long long cells = std::min(T, bc.ncell - x0);
        v.push_back({cells * bc.nvel / bc.nch, BItem{i, x0, ch}});
      }
  }
  if (cudaMemcpy((void*)b->p.cases, b->cases.data(), sizeof(BCase) * b->ncases, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return bfail(b, DVM_ERR_CUDA, "cases upload");
  std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
  std::vector<BItem> items(v.size());
  for (size_t i = 0; i < v.size(); ++i) items[i] = v[i].second;
  if (b->p.items) cudaFree((void*)b->p.items);
  BItem* d = nullptr;
  if (cudaMalloc(&d, sizeof(BItem) * items.size()) != cudaSuccess) return bfail(b, DVM_ERR_OOM, "items");
  b->p.items = d;
  b->p.nitems = (int)items.size();
  return bcheck(b, cudaMemcpy(d, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice),
                "items upload");
}

template <typename TS, typename TC, bool HO>
void launch_b_kinetic_t(dvm_batch* b, cudaStream_t s) {
  if (b->n2d) k_b_kinetic<TS, TC, HO, true><<<b->blocks, b->threads, 0, s>>>(b->p);
  else k_b_kinetic<TS, TC, HO, false><<<b->blocks, b->threads, 0, s>>>(b->p);
}

template <typename TS, typename TC, bool HO>
const void* kinetic_fn(bool d2) {
  return d2 ? (const void*)k_b_kinetic<TS, TC, HO, true> : (const void*)k_b_kinetic<TS, TC, HO, false>;
}

int kinetic_blocks(dvm_batch* b) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool ho = b->scheme != DVM_FKS;
  const bool d2 = b->n2d > 0;
  const void* fn = b->precision == DVM_F64
                       ? (ho ? kinetic_fn<double, double, true>(d2) : kinetic_fn<double, double, false>(d2))
                   : b->precision == DVM_F32
                       ? (ho ? kinetic_fn<float, float, true>(d2) : kinetic_fn<float, float, false>(d2))
                       : (ho ? kinetic_fn<__nv_bfloat16, float, true>(d2)
                             : kinetic_fn<__nv_bfloat16, float, false>(d2));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, b->threads, 0);
  if (per < 1) per = 1;
  if (b->ctas_per_sm > 0 && b->ctas_per_sm < per) per = b->ctas_per_sm;
  return sms * per;
}

void launch_kinetic(dvm_batch* b, cudaStream_t s) {
  const bool ho = b->scheme != DVM_FKS;
  if (b->precision == DVM_F64) { if (ho) launch_b_kinetic_t<double, double, true>(b, s); else launch_b_kinetic_t<double, double, false>(b, s); }
  else if (b->precision == DVM_F32) { if (ho) launch_b_kinetic_t<float, float, true>(b, s); else launch_b_kinetic_t<float, float, false>(b, s); }
  else { if (ho) launch_b_kinetic_t<__nv_bfloat16, float, true>(b, s); else launch_b_kinetic_t<__nv_bfloat16, float, false>(b, s); }
}

template <typename TS, typename TW>
void launch_euler_t(dvm_batch* b, cudaStream_t s) {
  if (b->n2d && b->scheme != DVM_FKS) {
    if (b->scheme == DVM_HOFKS) k_b_euler2d<TW, true><<<b->n2d, kBE, 0, s>>>(b->p);
    else k_b_euler2d<TW, false><<<b->n2d, kBE, 0, s>>>(b->p);
  }
  if (b->n1d == 0) return;
  const size_t sm = b->euler_smem;
  if (b->scheme == DVM_FKS) k_b_euler<TS, TW, true, false, false><<<b->ncases, kBE, sm, s>>>(b->p);
  else if (b->split_euler) {
    if (b->scheme == DVM_HOFKS) k_b_euler<TS, TW, true, true, true><<<b->ncases, kBE, sm, s>>>(b->p);
    else k_b_euler<TS, TW, false, true, true><<<b->ncases, kBE, sm, s>>>(b->p);
  } else {
    if (b->scheme == DVM_HOFKS) k_b_euler<TS, TW, true, true, false><<<b->ncases, kBE, sm, s>>>(b->p);
    else k_b_euler<TS, TW, false, true, false><<<b->ncases, kBE, sm, s>>>(b->p);
  }
}

void launch_euler(dvm_batch* b, cudaStream_t s) {
  if (b->precision == DVM_F64) launch_euler_t<double, double>(b, s);
  else if (b->precision == DVM_F32) launch_euler_t<float, float>(b, s);
  else launch_euler_t<__nv_bfloat16, float>(b, s);
}

template <typename TS, typename TW>
void set_euler_attr_t(dvm_batch* b) {
  const int sm = (int)b->euler_smem;
  cudaFuncSetAttribute(k_b_euler<TS, TW, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_b_euler<TS, TW, true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_b_euler<TS, TW, false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_b_euler<TS, TW, true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_b_euler<TS, TW, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

void launch_finalize(dvm_batch* b, cudaStream_t s) {
  const unsigned nb = (unsigned)((b->ncells + kB - 1) / kB);
  const bool ho = b->scheme != DVM_FKS;
  if (b->precision == DVM_F64) { if (ho) k_b_finalize<double, true><<<nb, kB, 0, s>>>(b->p); else k_b_finalize<double, false><<<nb, kB, 0, s>>>(b->p); }
  else { if (ho) k_b_finalize<float, true><<<nb, kB, 0, s>>>(b->p); else k_b_finalize<float, false><<<nb, kB, 0, s>>>(b->p); }
}

void launch_prepare(dvm_batch* b, cudaStream_t s) {
  if (b->precision == DVM_F64) k_b_prepare<double><<<b->ncases, 128, 0, s>>>(b->p);
  else if (b->precision == DVM_F32) k_b_prepare<float><<<b->ncases, 128, 0, s>>>(b->p);
  else k_b_prepare<__nv_bfloat16><<<b->ncases, 128, 0, s>>>(b->p);
}

// One batched step.  The Euler sub-steps read only W = (1 - lambda) U^n and
// the kinetic pass only f and the parameters, so (except in timed steps) the
// Euler kernel runs on a forked high-priority stream beside the kinetic pass.
int enqueue(dvm_batch* b, cudaStream_t s, bool timed = false) {
  launch_prepare(b, s);
  const bool euler = b->scheme != DVM_FKS;
  const bool fork = euler && !timed;
  if (euler) {
    cudaStream_t es = s;
    if (fork) {
      cudaEventRecord(b->fork, s);
      cudaStreamWaitEvent(b->side, b->fork, 0);
      es = b->side;
    }
    launch_euler(b, es);
    if (fork) cudaEventRecord(b->join, b->side);
  }
  if (timed) cudaEventRecord(b->e0, s);
  launch_kinetic(b, s);
  if (timed) cudaEventRecord(b->e1, s);
  if (fork) cudaStreamWaitEvent(s, b->join, 0);
  launch_finalize(b, s);
  return bcheck(b, cudaGetLastError(), "batch launch");
}

void drop(dvm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

int ensure_graph(dvm_batch* b) {
  if (b->exec) return 0;
  int rc = bcheck(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "capture");
  if (rc) return rc;
  rc = enqueue(b, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (rc) return rc;
  if ((rc = bcheck(b, e, "end capture"))) return rc;
  b->graph = g;
  return bcheck(b, cudaGraphInstantiate(&b->exec, g, 0), "instantiate");
}

int bsync(dvm_batch* b) {
  int rc = bcheck(b, cudaMemcpyAsync(b->pinned, b->p.status, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "status");
  if (rc) return rc;
  if ((rc = bcheck(b, cudaStreamSynchronize(b->stream), "sync"))) return rc;
  if (*b->pinned) return bfail(b, *b->pinned, "device error in a batch case");
  return 0;
}

}  // namespace

extern "C" {

int dvm_batch_create(const dvm_config* cfgs, int ncases, void* cuda_stream, dvm_batch** out) {
  if (!cfgs || ncases < 1 || !out) return DVM_ERR_ARG;
  *out = nullptr;
  dvm_batch* b = new dvm_batch();
  b->ncases = ncases;
  b->precision = cfgs[0].precision;
  b->scheme = cfgs[0].scheme;
  b->stream = (cudaStream_t)cuda_stream;
  const size_t tw = b->precision == DVM_F64 ? 8 : 4;
  long long cells = 0, pts = 0, escr = 0;
  int ghost = 0;
  std::vector<double> lam;
  for (int i = 0; i < ncases; ++i) {
    Geom g;
    std::string msg;
    if (make_geom(&cfgs[i], &g, &msg) || g.d > 2 || cfgs[i].precision != b->precision ||
        cfgs[i].scheme != b->scheme || cfgs[i].scheme == DVM_HOFKS_WENO || cfgs[i].scheme == DVM_FKS_STRANG || cfgs[i].tau_field || (g.d == 1 && g.nx[0] > kMaxBatchNx) ||
        (g.d == 2 && (g.bc[0] != DVM_BC_PERIODIC || g.bc[1] != DVM_BC_PERIODIC ||
                      g.nc > kMaxBatchCells2D))) {
      delete b;
      return DVM_ERR_ARG;
    }
    BCase c{};
    c.d = g.d;
    c.nx = g.nx[0];
    c.ny = g.d == 2 ? g.nx[1] : 1;
    c.nv = g.nv[0];
    c.nvy = g.d == 2 ? g.nv[1] : 1;
    c.kmin = g.kmin[0];
    c.kminy = g.d == 2 ? g.kmin[1] : 0;
    c.ncell = c.nx * c.ny;
    c.nvel = c.nv * c.nvy;
    c.nch = 1;
    c.p = g.p;
    c.bc = g.bc[0];
    c.forced_sub = g.forced_sub;
    c.ghost_off = ghost;
    c.f_off = pts;
    c.c_off = cells;
    c.e_off = g.d == 2 ? escr : 0;
    c.dx = g.dx;
    c.dv = g.dv;
    c.dt = g.dt;
    c.w = g.w;
    double A[kMaxM * kMaxM];
    if (invert_moment_matrix(g, A)) { delete b; return DVM_ERR_ARG; }
    for (int j = 0; j < g.nm * g.nm; ++j) c.A[j] = A[j], c.Af[j] = (float)A[j];
    const double l = exp(-g.dt / cfgs[i].tau);
    if (!(cfgs[i].tau >= 0)) { delete b; return DVM_ERR_ARG; }
    c.all_free = l == 1.0;
    for (int x = 0; x < c.ncell; ++x) lam.push_back(l);
    b->cases.push_back(c);
    if (g.d == 1) {
      b->max_nx = std::max(b->max_nx, c.nx);
      ghost += 2 * c.nv;
      b->n1d += 1;
    } else {
      b->n2d += 1;
      b->nmb = 4;
      escr += 24LL * c.ncell;  // W0, W1 and the four split fluxes, 4 components each
    }
    cells += c.ncell;
    pts += (long long)c.ncell * c.nvel;
  }
  b->ncells = cells;
  b->npoints = pts;
  BPtrs& p = b->p;
  p.ncases = ncases;
  p.ncells = cells;
  p.scheme = b->scheme;
  p.nmb = b->nmb;
  const int nmb = b->nmb;
  const size_t es = b->precision == DVM_F64 ? 8 : (b->precision == DVM_F32 ? 4 : 2);
  const size_t tc = b->precision == DVM_F64 ? 8 : 4;
  std::vector<int> cell_case;
  for (int i = 0; i < ncases; ++i)
    for (int x = 0; x < b->cases[i].ncell; ++x) cell_case.push_back(i);
  int rc = 0;
  BCase* dcases = nullptr;
  int* dcc = nullptr;
  const int np = prm_rows(nmb - 2);
  rc |= balloc(b, &dcases, sizeof(BCase) * ncases);
  rc |= balloc(b, &dcc, sizeof(int) * cells);
  rc |= balloc(b, &p.F, es * pts);
  rc |= balloc(b, &p.ghost, es * (ghost > 0 ? ghost : 1));
  rc |= balloc(b, &p.U, 8 * nmb * cells);
  rc |= balloc(b, &p.lam, 8 * cells);
  rc |= balloc(b, &p.UE, 8 * nmb * cells);
  rc |= balloc(b, &p.UM, 8 * nmb * cells);
  rc |= balloc(b, &p.Us, 8 * nmb * cells);
  rc |= balloc(b, &p.acc, 8 * (size_t)kMaxChunks * 2 * nmb * cells);
  rc |= balloc(b, &p.escr, tw * (escr > 0 ? escr : 1));
  rc |= balloc(b, &p.prm, tc * np * cells);
  rc |= balloc(b, &p.eqp, 8 * np * cells);
  rc |= balloc(b, &p.msub, sizeof(int) * ncases);
  rc |= balloc(b, &p.alpha, sizeof(double) * ncases);
  rc |= balloc(b, &p.status, 256);
  int* dorder = nullptr;
  int* dorder2 = nullptr;
  rc |= balloc(b, &dorder, sizeof(int) * ncases);
  rc |= balloc(b, &dorder2, sizeof(int) * ncases);
  if (rc) { dvm_batch_destroy(b); return DVM_ERR_OOM; }
  p.order = dorder;
  p.order2 = dorder2;
  // Euler work of a case ~ cells x sub-steps ~ N_cells N_v (the sub-step
  // count grows as the velocity spacing shrinks): largest first
  std::vector<int> order(ncases);
  for (int i = 0; i < ncases; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return (long long)b->cases[a].ncell * b->cases[a].nvel > (long long)b->cases[c].ncell * b->cases[c].nvel;
  });
  std::vector<int> order2;
  for (int i : order)
    if (b->cases[i].d == 2) order2.push_back(i);
  order2.resize(ncases, 0);
  p.step = (long long*)((char*)p.status + 64);
  p.qcounter = (unsigned*)((char*)p.status + 128);
  p.cases = dcases;
  p.cell_case = dcc;
  p.cpt = b->cpt;
  if (cudaMemcpy(dcases, b->cases.data(), sizeof(BCase) * ncases, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dcc, cell_case.data(), sizeof(int) * cells, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p.lam, lam.data(), 8 * cells, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dorder, order.data(), sizeof(int) * ncases, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dorder2, order2.data(), sizeof(int) * ncases, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(p.status, 0, 256) != cudaSuccess || cudaMemset(p.U, 0, 8 * nmb * cells) != cudaSuccess ||
      cudaMemset(p.UE, 0, 8 * nmb * cells) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&b->pinned, 64) != cudaSuccess ||
      cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    dvm_batch_destroy(b);
    return DVM_ERR_CUDA;
  }
  {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, hi) != cudaSuccess) {
      cudaGetLastError();
      dvm_batch_destroy(b);
      return DVM_ERR_CUDA;
    }
  }
  // W0, W1 and, for the split-flux form, G+ and G- (3 rows each) per 1D case;
  // the split form only while that fits next to a second CTA per SM
  b->split_euler = 4 * 3 * (size_t)b->max_nx * tw <= 110 * 1024;
  b->euler_smem = (b->split_euler ? 4 : 2) * 3 * (size_t)std::max(b->max_nx, 1) * tw;
  if (b->precision == DVM_F64) set_euler_attr_t<double, double>(b);
  else if (b->precision == DVM_F32) set_euler_attr_t<float, float>(b);
  else set_euler_attr_t<__nv_bfloat16, float>(b);
  b->blocks = kinetic_blocks(b);
  if (build_items(b)) { dvm_batch_destroy(b); return DVM_ERR_CUDA; }
  *out = b;
  return 0;
}

void dvm_batch_destroy(dvm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  drop(b);
  if (b->p.items) cudaFree((void*)b->p.items);
  for (void* q : b->allocs) cudaFree(q);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->pinned) cudaFreeHost(b->pinned);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  b->rb.release();
  delete b;
}

const char* dvm_batch_last_error(const dvm_batch* b) { return b ? b->err.c_str() : "null batch"; }

int dvm_batch_sizes(const dvm_batch* b, long long* cells, long long* points) {
  if (!b) return DVM_ERR_ARG;
  if (cells) *cells = b->ncells;
  if (points) *points = b->npoints;
  return 0;
}

int dvm_batch_moment_rows(const dvm_batch* b, int* rows) {
  if (!b || !rows) return DVM_ERR_ARG;
  *rows = b->nmb;
  return 0;
}

int dvm_batch_set_state_moments(dvm_batch* b, const double* U, int on_device) {
  if (!b || !U) return DVM_ERR_ARG;
  if (b->status) return b->status;
  cudaStream_t s = b->stream;
  int rc = bcheck(b, cudaMemcpyAsync(b->p.U, U, 8 * (size_t)b->nmb * b->ncells,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
                  "upload");
  rc |= bcheck(b, cudaMemsetAsync(b->p.status, 0, 256, s), "memset");
  if (rc) return b->status;
  const unsigned nb = (unsigned)((b->ncells + kB - 1) / kB);
  if (b->precision == DVM_F64) k_b_cell_params<double><<<nb, kB, 0, s>>>(b->p, 0, 1);
  else k_b_cell_params<float><<<nb, kB, 0, s>>>(b->p, 0, 1);
  dim3 gi(64, b->ncases);
  if (b->precision == DVM_F64) k_b_init_f<double, double><<<gi, kB, 0, s>>>(b->p);
  else if (b->precision == DVM_F32) k_b_init_f<float, float><<<gi, kB, 0, s>>>(b->p);
  else k_b_init_f<__nv_bfloat16, float><<<gi, kB, 0, s>>>(b->p);
  if (b->precision == DVM_F64) k_b_cell_params<double><<<nb, kB, 0, s>>>(b->p, 1, 1);
  else k_b_cell_params<float><<<nb, kB, 0, s>>>(b->p, 1, 1);
  if ((rc = bcheck(b, cudaGetLastError(), "init launch"))) return rc;
  if ((rc = bsync(b))) return rc;
  b->state_set = true;
  return 0;
}

int dvm_batch_step_async(dvm_batch* b, int nsteps) {
  if (!b) return DVM_ERR_ARG;
  if (b->status) return b->status;
  if (!b->state_set) return bfail(b, DVM_ERR_STATE, "step before a state was set");
  int rc = ensure_graph(b);
  if (rc) return rc;
  for (int i = 0; i < nsteps; ++i)
    if ((rc = bcheck(b, cudaGraphLaunch(b->exec, b->stream), "graph launch"))) return rc;
  return 0;
}

int dvm_batch_sync_status(dvm_batch* b) {
  if (!b) return DVM_ERR_ARG;
  if (b->status) return b->status;
  return bsync(b);
}

int dvm_batch_step(dvm_batch* b, int nsteps) {
  const int rc = dvm_batch_step_async(b, nsteps);
  return rc ? rc : bsync(b);
}

int dvm_batch_moments(dvm_batch* b, double* out, int on_device) {
  if (!b || !out) return DVM_ERR_ARG;
  if (b->status) return b->status;
  int rc = bcheck(b, cudaMemcpyAsync(out, b->p.U, 8 * (size_t)b->nmb * b->ncells,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream),
                  "copy");
  return rc ? rc : bcheck(b, cudaStreamSynchronize(b->stream), "sync");
}

int dvm_batch_moments_async(dvm_batch* b, double* out, int on_device, long long* ticket) {
  if (!b || !out || !ticket) return DVM_ERR_ARG;
  if (b->status) return b->status;
  return bcheck(b, b->rb.issue(b->stream, b->p.U, (long long)b->nmb * b->ncells, b->p.status, out, on_device != 0,
                               ticket),
                "moments read-back");
}

int dvm_batch_moments_wait(dvm_batch* b, long long ticket) {
  if (!b) return DVM_ERR_ARG;
  if (b->status) return b->status;
  if (ticket < 0 || ticket >= b->rb.issued) return bfail(b, DVM_ERR_ARG, "read-back ticket not issued");
  int st = 0;
  int rc = bcheck(b, b->rb.wait(ticket, &st), "read-back wait");
  if (rc) return rc;
  return st ? bfail(b, st, "device error in a batch case") : 0;
}

int dvm_batch_get_f(dvm_batch* b, int icase, double* out) {
  if (!b || !out || icase < 0 || icase >= b->ncases) return DVM_ERR_ARG;
  if (b->status) return b->status;
  const long long npts = (long long)b->cases[icase].ncell * b->cases[icase].nvel;
  double* d = nullptr;
  int rc = bcheck(b, cudaMalloc(&d, 8 * npts), "staging");
  if (rc) return rc;
  const unsigned nb = (unsigned)((npts + kB - 1) / kB);
  if (b->precision == DVM_F64) k_b_materialize<double, double><<<nb, kB, 0, b->stream>>>(b->p, icase, d);
  else if (b->precision == DVM_F32) k_b_materialize<float, float><<<nb, kB, 0, b->stream>>>(b->p, icase, d);
  else k_b_materialize<__nv_bfloat16, float><<<nb, kB, 0, b->stream>>>(b->p, icase, d);
  rc = bcheck(b, cudaGetLastError(), "materialize");
  if (!rc) rc = bcheck(b, cudaMemcpyAsync(out, d, 8 * npts, cudaMemcpyDeviceToHost, b->stream), "copy");
  if (!rc) rc = bcheck(b, cudaStreamSynchronize(b->stream), "sync");
  cudaFree(d);
  return rc;
}

int dvm_batch_info(dvm_batch* b, long long* n, int* substeps, double* alpha) {
  if (!b) return DVM_ERR_ARG;
  if (b->status) return b->status;
  int rc = 0;
  if (n) rc |= bcheck(b, cudaMemcpyAsync(n, b->p.step, 8, cudaMemcpyDeviceToHost, b->stream), "copy");
  if (substeps) rc |= bcheck(b, cudaMemcpyAsync(substeps, b->p.msub, sizeof(int) * b->ncases, cudaMemcpyDeviceToHost, b->stream), "copy");
  if (alpha) rc |= bcheck(b, cudaMemcpyAsync(alpha, b->p.alpha, 8 * b->ncases, cudaMemcpyDeviceToHost, b->stream), "copy");
  rc |= bcheck(b, cudaStreamSynchronize(b->stream), "sync");
  return rc ? b->status : 0;
}

int dvm_batch_set_tiling(dvm_batch* b, int threads, int cells_per_thread, int vchunks, int ctas_per_sm) {
  if (!b || threads < 32 || threads > 1024 || (threads & 31) || cells_per_thread < 1 || cells_per_thread > 8 ||
      vchunks < 1 || vchunks > kMaxChunks || ctas_per_sm < 0 || ctas_per_sm > 32)
    return DVM_ERR_ARG;
  if (b->status) return b->status;
  b->threads = threads;
  b->cpt = cells_per_thread;
  b->vch = vchunks;
  b->ctas_per_sm = ctas_per_sm;
  b->p.cpt = cells_per_thread;
  b->blocks = kinetic_blocks(b);
  drop(b);
  return build_items(b);
}

int dvm_batch_kinetic_ms(dvm_batch* b, int nsteps, double* ms) {
  if (!b || !ms || nsteps < 1) return DVM_ERR_ARG;
  if (b->status) return b->status;
  if (!b->state_set) return bfail(b, DVM_ERR_STATE, "no state");
  double tot = 0.0;
  for (int i = 0; i < nsteps; ++i) {
    int rc = enqueue(b, b->stream, true);
    if (rc) return rc;
    if ((rc = bcheck(b, cudaEventSynchronize(b->e1), "sync"))) return rc;
    float t = 0.f;
    cudaEventElapsedTime(&t, b->e0, b->e1);
    tot += t;
  }
  *ms = tot / nsteps;
  return bsync(b);
}

int dvm_batch_autotune(dvm_batch* b, int* threads, int* cells_per_thread, int* vchunks, int* ctas_per_sm,
                       double* best_ms) {
  if (!b) return DVM_ERR_ARG;
  if (b->status) return b->status;
  if (!b->state_set) return bfail(b, DVM_ERR_STATE, "no state");
  // time the kinetic pass of each candidate launch on the current state, then
  // put f back: the pass rewrites f in place
  const size_t es = b->precision == DVM_F64 ? 8 : (b->precision == DVM_F32 ? 4 : 2);
  const size_t fb = es * (size_t)b->npoints;
  void* save = nullptr;
  int rc = bcheck(b, cudaMalloc(&save, fb), "autotune staging");
  if (rc) return rc;
  cudaStream_t s = b->stream;
  cudaMemcpyAsync(save, b->p.F, fb, cudaMemcpyDeviceToDevice, s);
  // the ghost pieces of this step (the queue is reset before every timing)
  launch_prepare(b, s);
  const int cand_t[3] = {64, 128, 256}, cand_c[2] = {1, 2}, cand_v[3] = {1, 2, 4}, cand_o[3] = {0, 2, 4};
  double best = 1e30;
  int bt = b->threads, bcpt = b->cpt, bv = b->vch, bo = b->ctas_per_sm;
  for (int ti : cand_t)
    for (int ci : cand_c)
      for (int vi : cand_v)
        for (int oi : cand_o) {
          if ((rc = dvm_batch_set_tiling(b, ti, ci, vi, oi))) break;
          float acc = 0.f;
          for (int r = 0; r < 3; ++r) {
            cudaMemcpyAsync(b->p.F, save, fb, cudaMemcpyDeviceToDevice, s);
            cudaMemsetAsync(b->p.qcounter, 0, sizeof(unsigned), s);
            cudaEventRecord(b->e0, s);
            launch_kinetic(b, s);
            cudaEventRecord(b->e1, s);
            cudaEventSynchronize(b->e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, b->e0, b->e1);
            if (r > 0) acc += t;
          }
          if (acc / 2 < best) {
            best = acc / 2;
            bt = ti;
            bcpt = ci;
            bv = vi;
            bo = oi;
          }
        }
  cudaMemcpyAsync(b->p.F, save, fb, cudaMemcpyDeviceToDevice, s);
  cudaStreamSynchronize(s);
  cudaFree(save);
  if (!rc) rc = dvm_batch_set_tiling(b, bt, bcpt, bv, bo);
  if (rc) return rc;
  if (threads) *threads = bt;
  if (cells_per_thread) *cells_per_thread = bcpt;
  if (vchunks) *vchunks = bv;
  if (ctas_per_sm) *ctas_per_sm = bo;
  if (best_ms) *best_ms = best;
  return bcheck(b, cudaGetLastError(), "autotune");
}

}  // extern "C"
