// dvm_learn.cu -- kernels of the learned regime path.
//
// A flagged cell is taken to be at equilibrium for one step: its f^n is
// E[U^n] and its lambda is 0, the lambda -> 0 form of HOFKS that Theorem 1
// (Section 4.3.1) identifies with the MUSCL solution of the Euler system.
// Per step, before the Euler part:
//   flags       features of U^n -> network -> flag = (prediction < thr), or
//               the caller's flags; never on lambda = 1 or vetoed cells
//   apply       flagged cells: lambda row 0, Maxwellian weight 1 (L and mu''
//               rescaled by 1 / (1 - lambda)), W = U^n; cells flagged before
//               and not now are listed for write-back
//   deep        (windowed pass only) cells whose every source is flagged
//   materialise listed cells get E[U^n] written into their pieces
// and, every k steps, after the Euler part and before the kinetic pass:
//   check       full one-step kinetic update of sampled flagged cells and
//               the true log10 non-equilibrium of its result
#include <math.h>

#include "dvm_internal.cuh"
#include "dvm_learn.cuh"
#include "dvm_math.cuh"
#include "dvm_mlp.cuh"
#include "dvm_tc.cuh"

namespace dvm {
namespace {

__device__ inline int bc_wrap(int t, int n, int bc) {
  if (t >= 0 && t < n) return t;
  if (bc == DVM_BC_PERIODIC) {
    const int r = t % n;
    return r < 0 ? r + n : r;
  }
  return t < 0 ? 0 : n - 1;
}

// ---------------------------------------------------------------- features

// The ten regime features of cell c.  Differences of neighbouring states are
// formed in FP64 from the FP64 moments (no cancellation in the feature), the
// rest in FP32:
//   ln rho_+ - ln rho_- = log1p((rho_+ - rho_-) / rho_-)
//   ln theta_+ - ln theta_- = log1p((P_+ rho_-^2 - P_- rho_+^2) / (P_- rho_+^2)),
//     P = 2 E rho - |rho u|^2 = d rho^2 theta
//   u_+ - u_- = ((rho u)_+ rho_- - (rho u)_- rho_+) / (rho_+ rho_-)
template <int D>
__device__ void cell_features(const Geom& g, const double* __restrict__ U, long long c, float tau,
                              float out[kNIn]) {
  constexpr int NM = D + 2;
  const long long nc = g.nc;
  int x[3];
  cell_coords<D>(g, c, x);
  const double r0 = U[c];
  double m0[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < D; ++j) m0[j] = U[(1 + j) * nc + c];
  const double E0 = U[(NM - 1) * nc + c];
  double P0 = 2.0 * E0 * r0;
#pragma unroll
  for (int j = 0; j < D; ++j) P0 -= m0[j] * m0[j];
  const float rho = (float)r0;
  const float theta = (float)P0 / ((float)D * rho * rho);
  const float inv2dx = (float)(0.5 / g.dx);
  float glr2 = 0.f, glt2 = 0.f, div = 0.f, dyux = 0.f, dxuy = 0.f;
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {
    int xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
    xp[dir] = bc_wrap(x[dir] + 1, g.nx[dir], g.bc[dir]);
    xm[dir] = bc_wrap(x[dir] - 1, g.nx[dir], g.bc[dir]);
    const long long cp = cell_index(g, xp), cm = cell_index(g, xm);
    const double rp = U[cp], rm = U[cm];
    double mp[3] = {0.0, 0.0, 0.0}, mm[3] = {0.0, 0.0, 0.0};
    double Pp = 2.0 * U[(NM - 1) * nc + cp] * rp, Pm = 2.0 * U[(NM - 1) * nc + cm] * rm;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      mp[j] = U[(1 + j) * nc + cp];
      mm[j] = U[(1 + j) * nc + cm];
      Pp -= mp[j] * mp[j];
      Pm -= mm[j] * mm[j];
    }
    const float lr = log1pf((float)(rp - rm) / (float)rm);
    const double num = Pp * rm * rm, den = Pm * rp * rp;
    const float lt = log1pf((float)(num - den) / (float)den);
    const float rr = (float)rp * (float)rm;
    float du[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < D; ++j) du[j] = (float)(mp[j] * rm - mm[j] * rp) / rr * inv2dx;
    glr2 = fmaf(lr * inv2dx, lr * inv2dx, glr2);
    glt2 = fmaf(lt * inv2dx, lt * inv2dx, glt2);
    div += du[dir];
    if (dir == 1) dyux = du[0];
    if (dir == 0 && D >= 2) dxuy = du[1];
  }
  const float st = sqrtf(fmaxf(theta, 0.f));
  const float kn[5] = {tau * st * sqrtf(glr2), tau * st * sqrtf(glt2), tau * fabsf(div),
                       tau * fabsf(dyux), tau * fabsf(dxuy)};
  out[0] = rho;
  out[1] = (float)(m0[0] / r0);
  out[2] = D >= 2 ? (float)(m0[1] / r0) : 0.f;
  out[3] = theta;
  out[4] = log10f(tau);
#pragma unroll
  for (int j = 0; j < 5; ++j) out[5 + j] = log10f(fmaxf(kn[j], 1e-12f));
}

constexpr int kFlagBlock = 128;

// flags of step n from U^n (mode: DVM_LEARN_GIVEN or DVM_LEARN_MLP)
template <int D>
__global__ void __launch_bounds__(kFlagBlock) k_learn_flags(Geom g, DevPtrs p, LearnDev L, int mode,
                                                            float thr) {
  __shared__ __align__(16) float sP[kNP + 3];
  __shared__ float sN[2 * kNIn];
  __shared__ unsigned int cnt;
  const int tid = threadIdx.x;
  if (mode == DVM_LEARN_MLP) {
    for (int i = tid; i < kNP; i += kFlagBlock) sP[i] = L.P[i];
    if (tid < 2 * kNIn) sN[tid] = L.norm[tid];
  }
  if (tid == 0) cnt = 0u;
  __syncthreads();
  const long long c = blockIdx.x * (long long)kFlagBlock + tid;
  unsigned char fl = 0;
  if (c < g.nc) {
    float pred = 0.f;
    if (mode == DVM_LEARN_MLP) {
      float x[kNIn];
      cell_features<D>(g, p.U, c, L.tauf[c], x);
#pragma unroll
      for (int i = 0; i < kNIn; ++i) x[i] = (x[i] - sN[i]) * sN[kNIn + i];
      pred = mlp_forward_f32(sP, x);
      fl = pred < thr;
      L.pred[c] = pred;
    } else {
      fl = L.given[c] != 0;
    }
    fl = fl && p.lam[c] != 1.0 && !L.veto[c];
    L.flag_prev[c] = L.flag[c];
    L.flag[c] = fl;
  }
  const unsigned b = __ballot_sync(0xffffffffu, fl);
  if ((tid & 31) == 0 && b) atomicAdd(&cnt, (unsigned)__popc(b));
  __syncthreads();
  if (tid == 0 && cnt) atomicAdd(&L.cnt[kCntFlagged], (unsigned long long)cnt);
}

// MLP mode with the BF16 tensor-core network: 128 cells per tile, features in
// FP32 per thread, the two hidden layers as tcgen05 MMAs (FP32 accumulate)
template <int D>
__global__ void __launch_bounds__(tc::kTcThreads) k_learn_flags_tc(Geom g, DevPtrs p, LearnDev L, float thr) {
  __shared__ __align__(1024) tc::MlpSmem S;
  __shared__ float sN[2 * kNIn];
  __shared__ unsigned int cnt;
  const int tid = threadIdx.x;
  if (tid < 2 * kNIn) sN[tid] = L.norm[tid];
  if (tid == 0) cnt = 0u;
  tc::mlp_tc_setup(S, L.P);
  unsigned phase = 0;
  const long long ntiles = (g.nc + 127) / 128;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long c = tile * 128 + tid;
    const bool real = c < g.nc;
    float x[kNIn];
    if (real) {
      cell_features<D>(g, p.U, c, L.tauf[c], x);
#pragma unroll
      for (int i = 0; i < kNIn; ++i) x[i] = (x[i] - sN[i]) * sN[kNIn + i];
    } else {
#pragma unroll
      for (int i = 0; i < kNIn; ++i) x[i] = 0.f;
    }
    float pred = 0.f;
    if (!tc::mlp_tc_tile(S, phase, x, pred)) {
      if (tid == 0) set_status(p.status, DVM_ERR_TIMEOUT);
      break;
    }
    unsigned char fl = 0;
    if (real) {
      fl = pred < thr && p.lam[c] != 1.0 && !L.veto[c];
      L.pred[c] = pred;
      L.flag_prev[c] = L.flag[c];
      L.flag[c] = fl;
    }
    const unsigned b = __ballot_sync(0xffffffffu, fl);
    if ((tid & 31) == 0 && b) atomicAdd(&cnt, (unsigned)__popc(b));
  }
  tc::mlp_tc_teardown(S);
  if (tid == 0 && cnt) atomicAdd(&L.cnt[kCntFlagged], (unsigned long long)cnt);
}

// flagged cells: lambda 0, Maxwellian weight 1, W = U^n; cells that were
// flagged and are not any more are listed for write-back
template <typename TC, typename TW, int D>
__global__ void k_learn_apply(Geom g, DevPtrs p, LearnDev L) {
  constexpr int NM = D + 2;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  const long long nc = g.nc;
  if (L.flag[c]) {
    TC* prm = (TC*)p.prm;
    prm[prm_at(row_lam(), c, nc)] = TC(0);
    prm[prm_at(row_L(), c, nc)] += (TC)L.lw[c];
    const TC s = (TC)L.invw[c];
#pragma unroll
    for (int i = 0; i < NM; ++i) prm[prm_at(row_mu(D, i), c, nc)] *= s;
    if (g.scheme != DVM_FKS && !g.skip_euler) {
#pragma unroll
      for (int i = 0; i < NM; ++i) ((TW*)p.W0)[i * nc + c] = (TW)p.U[i * nc + c];
    }
  } else if (L.flag_prev[c]) {
    const unsigned i = atomicAdd(L.mat_count, 1u);
    L.mat_list[i] = (int)c;
  }
}

// out[c] = in[c - delta e_axis] true for every delta of the step along axis
// (p = 1: delta = k, k over the velocity indices): applied along every axis
// in turn to the flags it gives the cells whose whole source box is flagged
__global__ void k_learn_deep_axis(Geom g, const unsigned char* __restrict__ in,
                                  unsigned char* __restrict__ out, int axis) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  int x[3] = {(int)(c % g.nx[0]), (int)((c / g.nx[0]) % g.nx[1]),
              (int)(c / ((long long)g.nx[0] * g.nx[1]))};
  const int N = g.nx[axis];
  const long long stride = axis == 0 ? 1 : (axis == 1 ? g.nx[0] : (long long)g.nx[0] * g.nx[1]);
  const long long base = c - (long long)x[axis] * stride;
  unsigned char ok = 1;
  for (int k = g.kmin[axis]; k < g.kmin[axis] + g.nv[axis] && ok; ++k) {
    const int t = bc_wrap(x[axis] - k, N, g.bc[axis]);
    ok = in[base + (long long)t * stride];
  }
  out[c] = ok;
}

// E_k[U^n] into the pieces of the listed cells (their nu' is 0: the end of
// the step zeroes it for flagged cells, so the stored value is f itself)
template <typename TS, typename TC, int D>
__global__ void k_learn_materialise(Geom g, DevPtrs p, LearnDev L) {
  const unsigned cnt = *L.mat_count;
  if (blockIdx.x == 0 && threadIdx.x == 0 && cnt)
    atomicAdd(&L.cnt[kCntMaterialised], (unsigned long long)cnt);
  const long long total = (long long)cnt * g.nvel;
  const long long n = *p.step, nc = g.nc;
  const TC* prm = (const TC*)p.prm;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = L.mat_list[idx % cnt];
    const long long k = idx / cnt;
    int x[3];
    cell_coords<D>(g, c, x);
    const int kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
                       (int)(k / ((long long)g.nv[0] * g.nv[1]))};
    int q[3] = {0, 0, 0};
    TC qq = TC(0), vv = TC(0), lin = prm[prm_at(row_mu(D, 0), c, nc)];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const long long kg = g.kmin[i] + kk[i];
      q[i] = wrap((long long)x[i] - transport_offset(kg, n, g.p), g.nx[i]);
      const TC v = (TC)((double)kg * g.dv);
      const TC du = v - prm[prm_at(row_u(i), c, nc)];
      qq += du * du;
      vv += v * v;
      lin += prm[prm_at(row_mu(D, 1 + i), c, nc)] * v;
    }
    lin += prm[prm_at(row_mu(D, D + 1), c, nc)] * vv;
    const TC e = prm[prm_at(row_L(), c, nc)] - prm[prm_at(row_h(D), c, nc)] * qq;
    const TC M = sizeof(TC) == 8 ? (TC)exp2((double)e) : (TC)exp2f((float)e);
    const TC f = (M + lin) * (TC)L.invw[c];
    StoreT<TS>::store((TS*)p.F + k * nc + cell_index(g, q), f);
  }
}

__device__ inline unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// f*_k of cell x for velocity k: the same expression as the kinetic pass,
// lambda_s (F + nu'.m) + (M_s + mu''.m) with the source's (possibly
// flag-modified) parameters; returns a = the lambda part, b = the rest.
template <typename TS, typename TC, int D>
__device__ void fstar_of(const Geom& g, const DevPtrs& p, const int x[3], long long k, TC& a, TC& b,
                         TC v[3], TC& vv) {
  const long long n = *p.step, nc = g.nc;
  const int kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
                     (int)(k / ((long long)g.nv[0] * g.nv[1]))};
  int s[3] = {0, 0, 0}, q[3] = {0, 0, 0};
  bool clamped = false;
  vv = TC(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const long long kg = g.kmin[i] + kk[i];
    const long long o1 = transport_offset(kg, n + 1, g.p), o0 = transport_offset(kg, n, g.p);
    const int N = g.nx[i];
    long long t = x[i] - (o1 - o0);
    if (g.bc[i] == DVM_BC_PERIODIC) {
      t = wrap(t, N);
    } else if (t < 0 || t >= N) {
      t = t < 0 ? 0 : N - 1;
      clamped = true;
    }
    s[i] = (int)t;
    q[i] = wrap((long long)x[i] - o1, N);
    v[i] = (TC)((double)kg * g.dv);
    vv += v[i] * v[i];
  }
  const long long src = cell_index(g, s);
  TC fv;
  if (!clamped) {
    fv = StoreT<TS>::load((const TS*)p.F + k * nc + cell_index(g, q));
  } else if (g.ghost_mode == 1) {
    fv = StoreT<TS>::load((const TS*)p.ghost + 2 * k + (s[0] == 0 ? 0 : 1));
  } else {
    int qs[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const long long kg = g.kmin[i] + kk[i];
      qs[i] = wrap((long long)s[i] - transport_offset(kg, n, g.p), g.nx[i]);
    }
    fv = StoreT<TS>::load((const TS*)p.ghost + k * nc + cell_index(g, qs));
  }
  const TC* prm = (const TC*)p.prm;
  TC qq = TC(0), lmu = prm[prm_at(row_mu(D, 0), src, nc)], lnu = prm[prm_at(row_nu(D, 0), src, nc)];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const TC du = v[i] - prm[prm_at(row_u(i), src, nc)];
    qq += du * du;
    lmu += prm[prm_at(row_mu(D, 1 + i), src, nc)] * v[i];
    lnu += prm[prm_at(row_nu(D, 1 + i), src, nc)] * v[i];
  }
  lmu += prm[prm_at(row_mu(D, D + 1), src, nc)] * vv;
  lnu += prm[prm_at(row_nu(D, D + 1), src, nc)] * vv;
  const TC e = prm[prm_at(row_L(), src, nc)] - prm[prm_at(row_h(D), src, nc)] * qq;
  const TC M = sizeof(TC) == 8 ? (TC)exp2((double)e) : (TC)exp2f((float)e);
  a = prm[prm_at(row_lam(), src, nc)] * (fv + lnu);
  b = M + lmu;
}

constexpr int kCheckBlock = 128;

template <int N>
__device__ void block_sum(double v[N], double (*red)[kCheckBlock / 32]) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    double t = v[j];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = t;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N; ++j) {
    double t = 0.0;
    for (int w = 0; w < kCheckBlock / 32; ++w) t += red[j][w];
    v[j] = t;
  }
  __syncthreads();
}

// One-step check of cell c (one CTA): the full HOFKS update of the step from
// its sources (flagged ones at equilibrium), U^{n+1} = U_* + U_E, and the
// true log10 non-equilibrium of f^{n+1} = f* + m.nu against E[U^{n+1}].
template <typename TS, typename TC, typename TW, int D>
__global__ void __launch_bounds__(kCheckBlock) k_learn_check(Geom g, DevPtrs p, LearnDev L,
                                                             int explicit_cells, float thr,
                                                             int radius,
                                                             unsigned long long seed, int mlp) {
  constexpr int NM = D + 2;
  __shared__ double red[2 * kMaxM][kCheckBlock / 32];
  const long long nc = g.nc;
  long long c;
  if (explicit_cells) {
    c = L.check_cells[blockIdx.x];
  } else {
    const unsigned long long h = mix64(seed ^ mix64((unsigned long long)*p.step * 0x9e3779b97f4a7c15ull +
                                                    blockIdx.x));
    c = (long long)(h % (unsigned long long)nc);
    if (!L.flag[c]) return;
  }
  int x[3];
  cell_coords<D>(g, c, x);
  double acc[2 * kMaxM];
#pragma unroll
  for (int j = 0; j < 2 * NM; ++j) acc[j] = 0.0;
  for (long long k = threadIdx.x; k < g.nvel; k += kCheckBlock) {
    TC a, b, v[3], vv;
    fstar_of<TS, TC, D>(g, p, x, k, a, b, v, vv);
    const double m[kMaxM] = {1.0, (double)v[0], (double)v[1], (double)v[2], 0.0};
    acc[0] += (double)a;
    acc[NM] += (double)b;
#pragma unroll
    for (int i = 0; i < D; ++i) acc[1 + i] += (double)a * m[1 + i], acc[NM + 1 + i] += (double)b * m[1 + i];
    acc[NM - 1] += (double)a * 0.5 * (double)vv;
    acc[2 * NM - 1] += (double)b * 0.5 * (double)vv;
  }
  block_sum<2 * NM>(acc, red);
  // nu = A (U_E - U_M), U^{n+1} = U_* + U_E
  const TW* UE = (const TW*)((*p.msub & 1) ? p.W1 : p.W0);
  double r[kMaxM], Un[kMaxM], nu[kMaxM];
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    const double ue = g.skip_euler ? 0.0 : (double)UE[i * nc + c];
    r[i] = ue - g.w * acc[NM + i];
    Un[i] = g.w * acc[i] + ue;
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < NM; ++j) s += p.A[i * NM + j] * r[j];
    nu[i] = s;
  }
  double mu[kMaxM], rho, u[3], theta;
  const int rc = cell_mu<D>(g, p.A, Un, mu, rho, u, theta);
  double sums[2] = {0.0, 0.0};
  if (rc == 0) {
    const double pref = rho * pow(2.0 * M_PI * theta, -0.5 * D);
    for (long long k = threadIdx.x; k < g.nvel; k += kCheckBlock) {
      TC a, b, v[3], vv;
      fstar_of<TS, TC, D>(g, p, x, k, a, b, v, vv);
      double lin_nu = nu[0] + nu[NM - 1] * 0.5 * (double)vv, lin_mu = mu[0] + mu[NM - 1] * 0.5 * (double)vv;
      double q2 = 0.0;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        lin_nu += nu[1 + i] * (double)v[i];
        lin_mu += mu[1 + i] * (double)v[i];
        const double du = (double)v[i] - u[i];
        q2 += du * du;
      }
      const double f = (double)a + (double)b + g.w * lin_nu;
      const double E = pref * exp(-0.5 * q2 / theta) + g.w * lin_mu;
      sums[0] += fabs(f - E);
      sums[1] += fabs(E);
    }
  }
  block_sum<2>(sums, red);
  if (threadIdx.x != 0) return;
  const double ratio = rc ? 1.0 : sums[0] / sums[1];
  const float val = (float)log10(ratio > 1e-12 ? ratio : 1e-12);
  if (explicit_cells) L.check_out[blockIdx.x] = val;
  if (!L.flag[c]) return;
  atomicAdd(&L.cnt[kCntChecked], 1ull);
  if (mlp) {
    const double e = fabs((double)L.pred[c] - (double)val);
    atomicAdd(&L.err[0], e);
    atomicMax((unsigned long long*)&L.err[1], (unsigned long long)__double_as_longlong(e));
  }
  const double vt = (double)val + 12.0;  // >= 0: order of the bits is the order of the values
  atomicMax((unsigned long long*)&L.err[2], (unsigned long long)__double_as_longlong(vt));
  if (!(val < thr)) {
    atomicAdd(&L.cnt[kCntFailed], 1ull);
    const int rz = D == 3 ? radius : 0, ry = D >= 2 ? radius : 0;
    for (int dz = -rz; dz <= rz; ++dz)
      for (int dy = -ry; dy <= ry; ++dy)
        for (int dx = -radius; dx <= radius; ++dx) {
          const int y[3] = {bc_wrap(x[0] + dx, g.nx[0], g.bc[0]),
                            D >= 2 ? bc_wrap(x[1] + dy, g.nx[1], g.bc[1]) : 0,
                            D == 3 ? bc_wrap(x[2] + dz, g.nx[2], g.bc[2]) : 0};
          L.veto[cell_index(g, y)] = 1;
        }
  }
}

// every flagged cell onto the write-back list, flags cleared (the learned
// path is switched off or the state saved: f = E[U] goes into the pieces)
__global__ void k_learn_flush_list(Geom g, LearnDev L) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  if (L.flag[c]) L.mat_list[atomicAdd(L.mat_count, 1u)] = (int)c;
  L.flag[c] = 0;
  L.flag_prev[c] = 0;
}

// features of every cell, sample-major
template <int D>
__global__ void k_features(Geom g, DevPtrs p, LearnDev L, float* out) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  float x[kNIn];
  cell_features<D>(g, p.U, c, L.tauf[c], x);
#pragma unroll
  for (int i = 0; i < kNIn; ++i) out[c * kNIn + i] = x[i];
}

// log10(max(||f - E[U]||_1 / ||E[U]||_1, 1e-12)) per cell, in FP64 from the
// true f (stored piece + deferred term, or E for a flagged cell)
template <typename TS, typename TC, int D>
__global__ void k_noneq(Geom g, DevPtrs p, float* out) {
  constexpr int NM = D + 2;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  const long long nc = g.nc, n = *p.step;
  double Uc[kMaxM], mu[kMaxM], rho, u[3], theta;
#pragma unroll
  for (int i = 0; i < NM; ++i) Uc[i] = p.U[i * nc + c];
  if (cell_mu<D>(g, p.A, Uc, mu, rho, u, theta)) {
    out[c] = 0.f;
    return;
  }
  const bool flagged = g.learn && p.lflag[c];
  const double pref = rho * pow(2.0 * M_PI * theta, -0.5 * D);
  const TC* prm = (const TC*)p.prm;
  int x[3];
  cell_coords<D>(g, c, x);
  double num = 0.0, den = 0.0;
  for (long long k = 0; k < g.nvel; ++k) {
    const int kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
                       (int)(k / ((long long)g.nv[0] * g.nv[1]))};
    int q[3] = {0, 0, 0};
    double v[3] = {0.0, 0.0, 0.0}, vv = 0.0, q2 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const long long kg = g.kmin[i] + kk[i];
      q[i] = wrap((long long)x[i] - transport_offset(kg, n, g.p), g.nx[i]);
      v[i] = (double)kg * g.dv;
      vv += v[i] * v[i];
      q2 += (v[i] - u[i]) * (v[i] - u[i]);
    }
    double lin_mu = mu[0] + mu[NM - 1] * 0.5 * vv;
#pragma unroll
    for (int i = 0; i < D; ++i) lin_mu += mu[1 + i] * v[i];
    const double E = pref * exp(-0.5 * q2 / theta) + g.w * lin_mu;
    double f;
    if (flagged) {
      f = E;
    } else {
      f = (double)StoreT<TS>::load((const TS*)p.F + k * nc + cell_index(g, q));
      if (g.scheme == DVM_FKS) {
        double qq = 0.0, lin = (double)prm[prm_at(row_mu(D, 0), c, nc)];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const double du = v[i] - (double)prm[prm_at(row_u(i), c, nc)];
          qq += du * du;
          lin += (double)prm[prm_at(row_mu(D, 1 + i), c, nc)] * v[i];
        }
        lin += (double)prm[prm_at(row_mu(D, D + 1), c, nc)] * vv;
        f += exp2((double)prm[prm_at(row_L(), c, nc)] - (double)prm[prm_at(row_h(D), c, nc)] * qq) + lin;
      } else {
        double lin = (double)prm[prm_at(row_nu(D, 0), c, nc)];
#pragma unroll
        for (int i = 0; i < D; ++i) lin += (double)prm[prm_at(row_nu(D, 1 + i), c, nc)] * v[i];
        lin += (double)prm[prm_at(row_nu(D, D + 1), c, nc)] * vv;
        f += lin;
      }
    }
    num += fabs(f - E);
    den += fabs(E);
  }
  const double ratio = num / den;
  out[c] = (float)log10(ratio > 1e-12 ? ratio : 1e-12);
}

inline unsigned blocks_of(long long n, int b) { return (unsigned)((n + b - 1) / b); }

#define DVM_LEARN_BY_DIM(g, CALL) \
  do {                            \
    if ((g).d == 1) {             \
      constexpr int DD = 1;       \
      CALL;                       \
    } else if ((g).d == 2) {      \
      constexpr int DD = 2;       \
      CALL;                       \
    } else {                      \
      constexpr int DD = 3;       \
      CALL;                       \
    }                             \
  } while (0)

}  // namespace

void learn_launch_flags(const Geom& g, const DevPtrs& p, const LearnDev& L, int mode,
                        int mlp_precision, float thr, cudaStream_t s) {
  if (mode == DVM_LEARN_MLP && mlp_precision == DVM_BF16S) {
    const long long tiles = (g.nc + 127) / 128;
    const unsigned grid = (unsigned)(tiles < 152 * 4 ? tiles : 152 * 4);
    DVM_LEARN_BY_DIM(g, (k_learn_flags_tc<DD><<<grid, tc::kTcThreads, 0, s>>>(g, p, L, thr)));
    return;
  }
  DVM_LEARN_BY_DIM(g, (k_learn_flags<DD><<<blocks_of(g.nc, kFlagBlock), kFlagBlock, 0, s>>>(g, p, L, mode, thr)));
}

void learn_launch_apply(const Geom& g, const DevPtrs& p, const LearnDev& L, cudaStream_t s) {
  const unsigned nb = blocks_of(g.nc, 256);
  if (g.precision == DVM_F64)
    DVM_LEARN_BY_DIM(g, (k_learn_apply<double, double, DD><<<nb, 256, 0, s>>>(g, p, L)));
  else
    DVM_LEARN_BY_DIM(g, (k_learn_apply<float, float, DD><<<nb, 256, 0, s>>>(g, p, L)));
}

void learn_launch_deep(const Geom& g, const LearnDev& L, cudaStream_t s) {
  const unsigned nb = blocks_of(g.nc, 256);
  // flag -> tmp (x) -> deep (y) [-> tmp (z) -> deep copy]
  if (g.d == 2) {
    k_learn_deep_axis<<<nb, 256, 0, s>>>(g, L.flag, L.tmp, 0);
    k_learn_deep_axis<<<nb, 256, 0, s>>>(g, L.tmp, L.deep, 1);
  } else if (g.d == 3) {
    k_learn_deep_axis<<<nb, 256, 0, s>>>(g, L.flag, L.deep, 0);
    k_learn_deep_axis<<<nb, 256, 0, s>>>(g, L.deep, L.tmp, 1);
    k_learn_deep_axis<<<nb, 256, 0, s>>>(g, L.tmp, L.deep, 2);
  } else {
    k_learn_deep_axis<<<nb, 256, 0, s>>>(g, L.flag, L.deep, 0);
  }
}

void learn_launch_materialise(const Geom& g, const DevPtrs& p, const LearnDev& L, cudaStream_t s) {
  const unsigned nb = 152 * 4;
  if (g.precision == DVM_F64)
    DVM_LEARN_BY_DIM(g, (k_learn_materialise<double, double, DD><<<nb, 256, 0, s>>>(g, p, L)));
  else if (g.precision == DVM_F32)
    DVM_LEARN_BY_DIM(g, (k_learn_materialise<float, float, DD><<<nb, 256, 0, s>>>(g, p, L)));
  else
    DVM_LEARN_BY_DIM(g, (k_learn_materialise<__nv_bfloat16, float, DD><<<nb, 256, 0, s>>>(g, p, L)));
}

void learn_launch_check(const Geom& g, const DevPtrs& p, const LearnDev& L, int ncheck,
                        bool explicit_cells, float thr, int radius, unsigned long long seed,
                        bool mlp, cudaStream_t s) {
  if (ncheck <= 0) return;
  const int ex = explicit_cells ? 1 : 0, ml = mlp ? 1 : 0;
  if (g.precision == DVM_F64)
    DVM_LEARN_BY_DIM(g, (k_learn_check<double, double, double, DD><<<ncheck, kCheckBlock, 0, s>>>(
                            g, p, L, ex, thr, radius, seed, ml)));
  else if (g.precision == DVM_F32)
    DVM_LEARN_BY_DIM(g, (k_learn_check<float, float, float, DD><<<ncheck, kCheckBlock, 0, s>>>(
                            g, p, L, ex, thr, radius, seed, ml)));
  else
    DVM_LEARN_BY_DIM(g, (k_learn_check<__nv_bfloat16, float, float, DD><<<ncheck, kCheckBlock, 0, s>>>(
                            g, p, L, ex, thr, radius, seed, ml)));
}

void learn_launch_features(const Geom& g, const DevPtrs& p, const LearnDev& L, float* out,
                           cudaStream_t s) {
  DVM_LEARN_BY_DIM(g, (k_features<DD><<<blocks_of(g.nc, 128), 128, 0, s>>>(g, p, L, out)));
}

void learn_launch_noneq(const Geom& g, const DevPtrs& p, float* out, cudaStream_t s) {
  const unsigned nb = blocks_of(g.nc, 128);
  if (g.precision == DVM_F64)
    DVM_LEARN_BY_DIM(g, (k_noneq<double, double, DD><<<nb, 128, 0, s>>>(g, p, out)));
  else if (g.precision == DVM_F32)
    DVM_LEARN_BY_DIM(g, (k_noneq<float, float, DD><<<nb, 128, 0, s>>>(g, p, out)));
  else
    DVM_LEARN_BY_DIM(g, (k_noneq<__nv_bfloat16, float, DD><<<nb, 128, 0, s>>>(g, p, out)));
}

void learn_launch_flush(const Geom& g, const DevPtrs& p, const LearnDev& L, cudaStream_t s) {
  cudaMemsetAsync(L.mat_count, 0, sizeof(unsigned), s);
  k_learn_flush_list<<<blocks_of(g.nc, 256), 256, 0, s>>>(g, L);
  learn_launch_materialise(g, p, L, s);
}

void learn_prepare(const Geom&) {}

}  // namespace dvm
