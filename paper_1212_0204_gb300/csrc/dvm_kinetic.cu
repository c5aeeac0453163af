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

#include "dvm_internal.cuh"

namespace dvm {
namespace {

constexpr int kThreads = 256;

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
  int kx = (int)(kb % g.nv[0]);
  int ky = D > 1 ? (int)((kb / g.nv[0]) % g.nv[1]) : 0;
  int kz = D > 2 ? (int)(kb / ((long long)g.nv[0] * g.nv[1])) : 0;

  const TC* prm = (const TC*)p.prm;
  TS* F = (TS*)p.F;
  const TS* G = (const TS*)p.ghost;
  const TC lam_c = prm[row_lam() * nc + c];

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
    // parameters of the source cell
    TC qq = TC(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const TC du = v[i] - prm[row_u(i) * nc + src];
      qq += du * du;
    }
    const TC M = fexp2<TC>(prm[row_L() * nc + src] - prm[row_h(D) * nc + src] * qq);
    TC lin_mu = prm[row_mu(D, 0) * nc + src] + prm[row_mu(D, D + 1) * nc + src] * vv;
#pragma unroll
    for (int i = 0; i < D; ++i) lin_mu += prm[row_mu(D, 1 + i) * nc + src] * v[i];
    TC fnew;
    if (HOFKS) {
      TC lin_nu = prm[row_nu(D, 0) * nc + src] + prm[row_nu(D, D + 1) * nc + src] * vv;
#pragma unroll
      for (int i = 0; i < D; ++i) lin_nu += prm[row_nu(D, 1 + i) * nc + src] * v[i];
      const TC a = prm[row_lam() * nc + src] * (fv + lin_nu);  // T(lambda f^n)
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
    StoreT<TS>::store(F + k * nc + slot, fnew);
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
  const long long blocks = (g.nc + kThreads - 1) / kThreads;
  const long long want = 152LL * 8;
  long long s = (want + blocks - 1) / blocks;
  const long long maxs = g.nvel / 16 > 0 ? g.nvel / 16 : 1;
  if (s > maxs) s = maxs;
  if (s > 64) s = 64;
  if (s < 1) s = 1;
  return (int)s;
}

void launch_kinetic_pass(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  if (g.precision == DVM_F64) launch_generic<double, double>(g, p, s);
  else if (g.precision == DVM_F32) launch_generic<float, float>(g, p, s);
  else launch_generic<__nv_bfloat16, float>(g, p, s);
}

}  // namespace dvm
