// dvm_linmom.cu -- moments of the transported moment-matching term of HOFKS
// for the 3D windowed kinetic pass (periodic grids, integer shifts p = 1).
//
// The pass writes f^{n+1} = T(lambda f^n) + T((1 - lambda) E^n) (Section
// 4.3.1) and needs both parts' moments, U_* and U_M (Eq. UK).  The second part
// of a piece is (1 - lambda_s) E_k[U_s] = M_k + mu''_s . mt(v_k) (Eq. minimMax
// with the weight folded in), s = c - k the cell the piece covered at t^n.
// The window pass keeps a single quadratic per source for the deferred term
// and mu''.mt together and sums the new value and M only; the moments of the
// mu''.mt part,
//   B_a(c) = sum_k m_a(v_k) mu''(c - k) . mt(v_k),
//   m = (1, v, |v|^2 / 2),  mt = (1, v, |v|^2)  (the row convention of mu''),
// come from here: every product m_a mt_b is a polynomial in v whose monomials
// factor over the axes, so B is a sum of box correlations of the five fields
// mu''_b, each computed as one 1D sum of N_v1 taps per axis (work N_c 3 N_v1
// per monomial instead of N_c N_v): x-sums of the fields (17 arrays), y-sums
// of those (32 arrays), then z-sums combined into B (46 terms).  Then
// U_M = sum_k m_k M_k + B and U_* = sum_k m_k f^{n+1} - U_M; the last velocity
// split of the partial sums holds (-B, +B), so the end-of-step kernel adds it
// like any other split.
#include <map>
#include <tuple>
#include <type_traits>
#include <vector>

#include "dvm_internal.cuh"

namespace dvm {
namespace {

constexpr int kLinMaxArr = 40;   // 17 x-sums, 32 y-sums
constexpr int kLinMaxTerm = 48;  // 46 terms
constexpr int kLinQ = 32;        // axis positions per CTA of the staged passes
constexpr int kLinWarps = 8;

// One pass: per input array i, its 1D sums with the powers 0..pmax[i] of the
// axis velocity, and the entries [beg[i], end[i]): in the x and y passes
// output array `out` = the sum with power pw; in the last pass, moment a +=
// coef * (the sum with power pw).
struct LinPass {
  int nin;
  signed char src[kLinMaxArr], pmax[kLinMaxArr];
  unsigned char beg[kLinMaxArr], end[kLinMaxArr];
  signed char pw[kLinMaxTerm], out[kLinMaxTerm];
  float coef[kLinMaxTerm];
};

struct LinTables {
  LinPass x;      // fields mu''_b -> x-sums
  LinPass y;      // x-sums -> xy-sums
  LinPass last;   // xy-sums along z -> B
  int nx, ny;     // arrays written by the x and y passes
};

// The monomials of m_a mt_b, grouped into the passes.
LinTables make_tables() {
  constexpr int d = 3;
  using Mono = std::tuple<int, int, int>;
  auto poly_m = [](int a) {
    std::map<Mono, double> r;
    if (a == 0) r[{0, 0, 0}] = 1.0;
    else if (a <= d) r[{a == 1, a == 2, a == 3}] = 1.0;
    else for (int i = 0; i < d; ++i) r[{2 * (i == 0), 2 * (i == 1), 2 * (i == 2)}] = 0.5;
    return r;
  };
  auto poly_mt = [](int b) {
    std::map<Mono, double> r;
    if (b == 0) r[{0, 0, 0}] = 1.0;
    else if (b <= d) r[{b == 1, b == 2, b == 3}] = 1.0;
    else for (int i = 0; i < d; ++i) r[{2 * (i == 0), 2 * (i == 1), 2 * (i == 2)}] = 1.0;
    return r;
  };
  const int nm = d + 2;
  // (b, px, py, pz, a) -> coefficient
  std::map<std::tuple<int, int, int, int, int>, double> terms;
  for (int a = 0; a < nm; ++a)
    for (int b = 0; b < nm; ++b)
      for (const auto& [m1, c1] : poly_m(a))
        for (const auto& [m2, c2] : poly_mt(b))
          terms[{b, std::get<0>(m1) + std::get<0>(m2), std::get<1>(m1) + std::get<1>(m2),
                 std::get<2>(m1) + std::get<2>(m2), a}] += c1 * c2;
  LinTables T{};
  // grouped entries of one pass: input -> list of (power, out, coef)
  auto fill = [](LinPass& P, const std::vector<std::vector<std::tuple<int, int, double>>>& by_in,
                 const std::vector<int>& src) {
    P.nin = (int)by_in.size();
    int ne = 0;
    for (int i = 0; i < P.nin; ++i) {
      P.src[i] = (signed char)src[i];
      P.beg[i] = (unsigned char)ne;
      int pmax = 0;
      for (const auto& [pw, out, c] : by_in[i]) {
        P.pw[ne] = (signed char)pw;
        P.out[ne] = (signed char)out;
        P.coef[ne] = (float)c;
        pmax = pw > pmax ? pw : pmax;
        ++ne;
      }
      P.end[i] = (unsigned char)ne;
      P.pmax[i] = (signed char)pmax;
    }
  };
  std::map<std::pair<int, int>, int> xi;        // (b, px) -> x-sum
  std::map<std::tuple<int, int, int>, int> yi;  // (b, px, py) -> xy-sum
  for (const auto& [k, c] : terms) xi.emplace(std::make_pair(std::get<0>(k), std::get<1>(k)), 0);
  {
    int n = 0;
    for (auto& [k, idx] : xi) idx = n++;
    T.nx = n;
    std::vector<std::vector<std::tuple<int, int, double>>> by_in(nm);
    std::vector<int> src(nm);
    for (int b = 0; b < nm; ++b) src[b] = b;
    for (const auto& [k, idx] : xi) by_in[k.first].emplace_back(k.second, idx, 1.0);
    fill(T.x, by_in, src);
  }
  {
    for (const auto& [k, c] : terms) yi.emplace(std::make_tuple(std::get<0>(k), std::get<1>(k), std::get<2>(k)), 0);
    int n = 0;
    for (auto& [k, idx] : yi) idx = n++;
    T.ny = n;
    std::vector<std::vector<std::tuple<int, int, double>>> by_in(T.nx);
    std::vector<int> src(T.nx);
    for (int j = 0; j < T.nx; ++j) src[j] = j;
    for (const auto& [k, idx] : yi)
      by_in[xi.at({std::get<0>(k), std::get<1>(k)})].emplace_back(std::get<2>(k), idx, 1.0);
    fill(T.y, by_in, src);
  }
  // terms by input array of the last pass
  std::vector<std::vector<std::tuple<int, int, double>>> by_in(T.ny);
  std::vector<int> src(T.ny);
  for (int i = 0; i < T.ny; ++i) src[i] = i;
  for (const auto& [k, c] : terms) {
    const auto [b, px, py, pz, a] = k;
    by_in[yi.at({b, px, py})].emplace_back(pz, a, c);
  }
  fill(T.last, by_in, src);
  return T;
}

const LinTables& tables() {
  static const LinTables t = make_tables();
  return t;
}

// velocities of one axis and their powers 0..4: s_vp[q * nv + t] = v_t^q
__device__ __forceinline__ void load_vpow(const Geom& g, int axis, float* s_vp) {
  const int nv = g.nv[axis];
  for (int t = threadIdx.x; t < nv; t += blockDim.x) {
    const float v = (float)((double)(g.kmin[axis] + t) * g.dv);
    float w = 1.f;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      s_vp[q * nv + t] = w;
      w *= v;
    }
  }
}

// the value sums with powers 0..PM of the axis velocity
template <int PM>
__device__ __forceinline__ void acc_powers(float* acc, const float* s_vp, int nv, int t, float v) {
  acc[0] += v;
#pragma unroll
  for (int w = 1; w <= PM; ++w) acc[w] = fmaf(s_vp[w * nv + t], v, acc[w]);
}

__device__ __forceinline__ float pick(const float* acc, int pw) {
  float val = acc[0];
#pragma unroll
  for (int w = 1; w < 5; ++w)
    if (pw == w) val = acc[w];
  return val;
}

// x-sums, one thread per (cell, field): all powers of v_x that field needs,
// the N_v1 sources of a cell read through L1 (neighbouring cells share them)
template <int PM>
__device__ __forceinline__ void lin_x_sums(const float* base, int s, int Nx, int nv, const float* s_vp,
                                           float* acc) {
  int t = 0;
  for (; t + 4 <= nv; t += 4) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = __ldg(base + 4 * s);
      if (--s < 0) s += Nx;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc_powers<PM>(acc, s_vp, nv, t + u, v[u]);
  }
  for (; t < nv; ++t) {
    acc_powers<PM>(acc, s_vp, nv, t, __ldg(base + 4 * s));
    if (--s < 0) s += Nx;
  }
}

__global__ void __launch_bounds__(256) k_lin_x(Geom g, DevPtrs p, LinPass P) {
  extern __shared__ float s_vp[];  // [5][nv]
  load_vpow(g, 0, s_vp);
  __syncthreads();
  const long long c = blockIdx.x * 256LL + threadIdx.x;
  if (c >= g.nc) return;
  const int i = blockIdx.y;
  const int Nx = g.nx[0], nv = g.nv[0];
  const int x = (int)(c % Nx);
  const float* prm = (const float*)p.prm;
  // cell (row start + s) of parameter row r sits at prm_at(r, row start) + 4 s
  const float* base = prm + prm_at(row_mu(3, P.src[i]), c - x, g.nc);
  const int s = wrap((long long)x - g.kmin[0], Nx);  // source of the first velocity
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  switch (P.pmax[i]) {
    case 0: lin_x_sums<0>(base, s, Nx, nv, s_vp, acc); break;
    case 1: lin_x_sums<1>(base, s, Nx, nv, s_vp, acc); break;
    case 2: lin_x_sums<2>(base, s, Nx, nv, s_vp, acc); break;
    case 3: lin_x_sums<3>(base, s, Nx, nv, s_vp, acc); break;
    default: lin_x_sums<4>(base, s, Nx, nv, s_vp, acc); break;
  }
  for (int e = P.beg[i]; e < P.end[i]; ++e) p.lin[(long long)P.out[e] * g.nc + c] = pick(acc, P.pw[e]);
}

__device__ __forceinline__ void cp_async_f4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_lin() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_lin() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One input of a staged pass: its sums with powers 0..PM for the QW positions
// of the thread, then its entries: x/y pass -> output arrays, last pass -> B.
template <int QW, int PM, int NM, bool LAST>
__device__ __forceinline__ void lin_body(const float* col, int nv, const float* s_vp, const LinPass& P, int i,
                                         float (&B)[QW][NM], float* lin, int out_off, long long nc,
                                         const long long (&q)[QW], bool xact) {
  float acc[QW][5];
#pragma unroll
  for (int j = 0; j < QW; ++j)
#pragma unroll
    for (int u = 0; u < 5; ++u) acc[j][u] = 0.f;
  for (int t = 0; t < nv; ++t) {
    const float* r = col - 32 * t;
#pragma unroll
    for (int j = 0; j < QW; ++j) acc_powers<PM>(acc[j], s_vp, nv, t, r[32 * kLinWarps * j]);
  }
  for (int e = P.beg[i]; e < P.end[i]; ++e) {
    const int pw = P.pw[e];
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      float val = acc[j][0];
#pragma unroll
      for (int u = 1; u <= PM; ++u)
        if (pw == u) val = acc[j][u];
      if constexpr (LAST) {
        const int a = P.out[e];
        const float cf = P.coef[e];
#pragma unroll
        for (int m = 0; m < NM; ++m)
          if (a == m) B[j][m] = fmaf(cf, val, B[j][m]);
      } else {
        if (xact && q[j] >= 0) lin[(long long)(out_off + P.out[e]) * nc + q[j]] = val;
      }
    }
  }
}

// The y and z axes: a CTA takes 32 consecutive x cells and
// kLinQ consecutive positions along the axis; per input array it stages the
// kLinQ + N_v1 - 1 source positions of its 32 columns in shared memory (one
// coalesced asynchronous copy per value), then warp w takes the positions w,
// w + kLinWarps, ...
// LAST = false: the y axis, one input per CTA, x-sums -> xy-sums (blockIdx.z =
// z * inputs + input; output arrays out_off + out).
// LAST = true: the z axis (blockIdx.z = y), all inputs in one CTA (the next
// input's slab copied while the current one is summed), the terms combined
// into B per cell, written to split `slice` of the partial sums as (-B, +B).
template <bool LAST>
__global__ void __launch_bounds__(32 * kLinWarps) k_lin_axis(Geom g, DevPtrs p, LinPass P, int in_off,
                                                             int out_off, int slice) {
  constexpr int NM = 5;
  const int axis = LAST ? 2 : 1;
  constexpr int QW = kLinQ / kLinWarps;  // positions per warp
  const int nv = g.nv[axis];
  const int rows = kLinQ + nv - 1;
  extern __shared__ float s_dyn[];
  float* s_vp = s_dyn;                     // [5][nv]
  float* s_slab = s_dyn + 5 * nv;          // [LAST ? 2 : 1][rows][32]
  load_vpow(g, axis, s_vp);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int Nx = g.nx[0];
  const int N = g.nx[axis];
  const long long stride = axis == 1 ? Nx : (long long)Nx * g.nx[1];
  const int xr = blockIdx.x * 32 + lane;
  const bool xact = xr < Nx;
  const int x = xact ? xr : Nx - 1;
  const int q0 = blockIdx.y * kLinQ;
  // offset of the remaining coordinate (z for the y pass, y for the z pass)
  long long other = 0;
  int i_beg = 0, i_end = P.nin;
  if (!LAST) {
    i_beg = (int)(blockIdx.z % P.nin);
    i_end = i_beg + 1;
    other = (long long)(blockIdx.z / P.nin) * Nx * g.nx[1];
  } else {
    other = (long long)blockIdx.z * Nx;
  }
  const int kmax = g.kmin[axis] + nv - 1;
  const int r0 = wrap((long long)q0 - kmax, N);  // staged row r: position (q0 - kmax + r) mod N
  auto stage = [&](int i, int buf) {
    const float* in = p.lin + (long long)(in_off + P.src[i]) * g.nc + other + x;
    float* dst = s_slab + (long long)buf * rows * 32 + lane;
    for (int r = w; r < rows; r += kLinWarps) {
      int q = r0 + r;
      if (q >= N) q %= N;
      cp_async_f4(dst + r * 32, in + (long long)q * stride);
    }
    cp_async_commit_lin();
  };
  float B[QW][NM];
#pragma unroll
  for (int j = 0; j < QW; ++j)
#pragma unroll
    for (int a = 0; a < NM; ++a) B[j][a] = 0.f;
  // cell offset of the warp's positions (-1 past the end of the axis)
  long long q[QW];
#pragma unroll
  for (int j = 0; j < QW; ++j) {
    const int qq = q0 + w + kLinWarps * j;
    q[j] = qq < N ? other + x + (long long)qq * stride : -1;
  }
  stage(i_beg, 0);
  for (int i = i_beg; i < i_end; ++i) {
    const int buf = LAST ? (i & 1) : 0;
    if (LAST && i + 1 < i_end) {
      stage(i + 1, buf ^ 1);
      cp_async_wait_lin<1>();
    } else {
      cp_async_wait_lin<0>();
    }
    __syncthreads();  // this input's slab (and s_vp) visible to all warps
    // position w + kLinWarps j, velocity t: staged row w + kLinWarps j + nv - 1 - t
    const float* col = s_slab + (long long)buf * rows * 32 + (w + nv - 1) * 32 + lane;
    switch (P.pmax[i]) {
      case 0: lin_body<QW, 0, NM, LAST>(col, nv, s_vp, P, i, B, p.lin, out_off, g.nc, q, xact); break;
      case 1: lin_body<QW, 1, NM, LAST>(col, nv, s_vp, P, i, B, p.lin, out_off, g.nc, q, xact); break;
      case 2: lin_body<QW, 2, NM, LAST>(col, nv, s_vp, P, i, B, p.lin, out_off, g.nc, q, xact); break;
      case 3: lin_body<QW, 3, NM, LAST>(col, nv, s_vp, P, i, B, p.lin, out_off, g.nc, q, xact); break;
      default: lin_body<QW, 4, NM, LAST>(col, nv, s_vp, P, i, B, p.lin, out_off, g.nc, q, xact); break;
    }
    if (LAST) __syncthreads();  // every warp done with this buffer before it is restaged
  }
  if (LAST && xact) {
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      if (q[j] < 0) continue;
      double* out = p.acc + (long long)slice * 2 * NM * g.nc + q[j];
#pragma unroll
      for (int a = 0; a < NM; ++a) {
        out[(long long)a * g.nc] = -(double)B[j][a];
        out[(long long)(NM + a) * g.nc] = (double)B[j][a];
      }
    }
  }
}

// dynamic shared memory: the velocity powers and one (two for the last pass)
// staged slabs of kLinQ + nv - 1 rows of 32 floats (LAST at 256 velocities:
// 78.6 KB, so the attribute is raised at creation)
size_t lin_axis_smem(int nv, bool last) {
  return sizeof(float) * (5 * (size_t)nv + (last ? 2 : 1) * 32 * (size_t)(kLinQ + nv - 1));
}

}  // namespace

// float arrays of the linear-term sums per cell (x-sums, then xy-sums)
int linear_moment_arrays() {
  const LinTables& T = tables();
  return T.nx + T.ny;
}

// B into the last split of the partial sums (see the top of this file); with
// the learned path (whose window pass sums both parts itself) that split is
// zero.  Returns the kernels launched.
int launch_linear_moments(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  constexpr int NM = 5;
  const int slice = g.nsplit - 1;
  if (g.learn) {
    cudaMemsetAsync(p.acc + (long long)slice * 2 * NM * g.nc, 0, sizeof(double) * 2 * NM * g.nc, s);
    return 0;
  }
  const LinTables& T = tables();
  const unsigned nb = (unsigned)((g.nc + 255) / 256);
  const unsigned bx = (unsigned)((g.nx[0] + 31) / 32);
  const unsigned by = (unsigned)((g.nx[1] + kLinQ - 1) / kLinQ);
  const unsigned bz = (unsigned)((g.nx[2] + kLinQ - 1) / kLinQ);
  k_lin_x<<<dim3(nb, T.x.nin), 256, sizeof(float) * 5 * g.nv[0], s>>>(g, p, T.x);
  // y pass: one input per CTA (blockIdx.z = z * inputs + input)
  k_lin_axis<false><<<dim3(bx, by, (unsigned)(g.nx[2] * T.y.nin)), 32 * kLinWarps, lin_axis_smem(g.nv[1], false),
                      s>>>(g, p, T.y, 0, T.nx, slice);
  // z pass: blockIdx.y = z block, blockIdx.z = y
  k_lin_axis<true><<<dim3(bx, bz, (unsigned)g.nx[1]), 32 * kLinWarps, lin_axis_smem(g.nv[2], true), s>>>(
      g, p, T.last, T.nx, 0, slice);
  return 3;
}

// Kernel attributes set before the first launch (outside any stream capture).
void linear_moments_prepare(const Geom& g) {
  cudaFuncSetAttribute(k_lin_axis<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lin_axis_smem(g.nv[1], false));
  cudaFuncSetAttribute(k_lin_axis<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lin_axis_smem(g.nv[2], true));
}

}  // namespace dvm
