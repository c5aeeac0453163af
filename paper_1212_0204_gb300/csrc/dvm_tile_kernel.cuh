// dvm_tile_kernel.cuh -- the 3D kinetic pass (HOFKS, single-quadratic form,
// periodic, integer shifts p = 1) for configured shapes, with the CTA's
// source rows folded once and shared.  Included by dvm_kinetic_shapes.cu.
//
// CTA = 4 warps stacked in y over 32 x cells and 16 y cells of one z plane;
// all four warps take the same velocity pair (kz, kx) at the same time.  For
// a pair, the sources of the CTA's targets over all ky are 16 + N_v1 - 1 rows
// of 32 cells, each folded with (vx, vz) into a 7-float slot (dvm_window.cuh,
// SlotP); the CTA folds them once into shared memory (each thread a quarter
// of a row's loads), then every thread slides its window of Y = 4 slots along
// ky reading one slot per step from shared memory.  Compared with the
// per-thread windows of dvm_window_kernel.cuh a source row is loaded and
// folded once per CTA instead of once per target thread (4x fewer parameter
// loads and folds), the parameter loads are not in the per-update dependency
// chain, and each warp owns its targets (no cross-warp moment reduction):
// the moment sums stay in registers, FP32 per pair and across the split's
// pairs, FP64 across splits.
#pragma once

#include "dvm_window_kernel.cuh"

namespace dvm {
namespace {

constexpr int kTileW = 4;                 // warps per CTA (stacked in y)
constexpr int kTileY = 4;                 // targets per thread (consecutive y)
constexpr int kTileTY = kTileW * kTileY;  // y cells per CTA

__host__ __device__ constexpr int tile_rows(int nv) { return kTileTY + nv - 1; }

// dynamic shared memory: the folded slots of one pair [rows][2][32] float4
// ((lambda, c0, c1, c2), (p0, p1, p2, -)) and the staged f of two blocks
// [2][Y][Y][128]
constexpr size_t tile_smem(int nv) {
  return sizeof(float) * (8 * (size_t)tile_rows(nv) * 32 + 2 * kTileY * kTileY * 32 * kTileW);
}

template <typename TS, int CX, int CY, int CZ, int CV>
__global__ void __launch_bounds__(32 * kTileW, 3) k_kpass_tile3(Geom g, DevPtrs p, int splits) {
  constexpr int Y = kTileY, NM = 5, NT = 2;
  constexpr int NT_ = 32 * kTileW;  // threads
  constexpr int ROWS = tile_rows(CV);
  static_assert(CX % 32 == 0 && CY % kTileTY == 0, "configured shapes tile exactly");
  __shared__ int s_ox[CV], s_oy[CV], s_oz[CV];
  extern __shared__ float4 s_tile_raw[];
  float4* s_slot = s_tile_raw;                               // [ROWS][2][32]
  float* s_fb = reinterpret_cast<float*>(s_tile_raw + 2 * ROWS * 32);  // [2][Y][Y][NT_]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long n1 = *p.step + 1;
  constexpr int Nx = CX, Ny = CY, Nz = CZ, nv = CV;
  constexpr long long nc = (long long)CX * CY * CZ;
  constexpr int plane = CX * CY;
  for (int t = tid; t < nv; t += NT_) {
    s_ox[t] = wrap((long long)(g.kmin[0] + t) * n1, Nx);
    s_oy[t] = wrap((long long)(g.kmin[1] + t) * n1, Ny);
    s_oz[t] = wrap((long long)(g.kmin[2] + t) * n1, Nz);
  }
  __syncthreads();
  const int x = blockIdx.x * 32 + lane;
  const int y0 = blockIdx.y * kTileTY;  // the CTA's first target row
  const int yw = y0 + w * Y;            // this warp's first target row
  const int z = (int)(blockIdx.z % Nz);
  const int split = (int)(blockIdx.z / Nz);
  const float dv = (float)g.dv;
  const float4* __restrict__ pg = (const float4*)p.wprm;
  TS* __restrict__ F = (TS*)p.F;
  const int npairs = nv * nv;
  const int per = npairs / splits;
  const int pb = split * per, pe = pb + per;
  constexpr long long kystep = (long long)nv * nc;
  // staged row r of a pair holds source row (y0 - (kmin_y + nv - 1) + r) mod Ny
  int r0 = (y0 - (g.kmin[1] + nv - 1)) % Ny;
  if (r0 < 0) r0 += Ny;

  // f of a block of Y steps x Y targets of pair pr_i from step kb_i down,
  // staged by cp.async (every address valid: rows wrapped)
  auto issue = [&](int pr_i, int kb_i, int st) {
    const int kx_i = pr_i % nv, kz_i = pr_i / nv;
    int qx_i = x - s_ox[kx_i];
    if (qx_i < 0) qx_i += Nx;
    int qz_i = z - s_oz[kz_i];
    if (qz_i < 0) qz_i += Nz;
    const TS* Fb_i = F + ((long long)kx_i + (long long)nv * nv * kz_i) * nc + qx_i + (long long)plane * qz_i;
    float* dst = s_fb + st * Y * Y * NT_ + tid;
#pragma unroll
    for (int jj = 0; jj < Y; ++jj) {
      int r = yw - s_oy[kb_i - jj];
      if (r < 0) r += Ny;
      const TS* Fk = Fb_i + (long long)(kb_i - jj) * kystep;
#pragma unroll
      for (int j = 0; j < Y; ++j) {
        cp_async4(dst + (jj * Y + j) * NT_, Fk + r * Nx);
        if (++r == Ny) r = 0;
      }
    }
  };

  float tot[NT][NM][Y];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int a = 0; a < NM; ++a)
#pragma unroll
      for (int j = 0; j < Y; ++j) tot[t][a][j] = 0.f;
  if (pb < pe) {
    issue(pb, nv - 1, 0);
    cp_async_commit();
  }
  int stage = 0;
  for (int pr = pb; pr < pe; ++pr) {
    const int kx = pr % nv, kz = pr / nv;
    const int kxg = g.kmin[0] + kx, kzg = g.kmin[2] + kz;
    const float vx = kxg * dv, vz = kzg * dv;
    const float vxz2 = fmaf(vx, vx, vz * vz);
    // ---- fold: this pair's source rows into the shared slots
    int sx = (x - kxg) % Nx;
    if (sx < 0) sx += Nx;
    int sz = (z - kzg) % Nz;
    if (sz < 0) sz += Nz;
    const int src_col = sx + plane * sz;
    __syncthreads();  // the previous pair's slots have been read
    for (int r = w; r < ROWS; r += kTileW) {
      int sr = r0 + r;
      if (sr >= Ny) sr -= Ny;
      if (sr >= Ny) sr -= Ny;
      const int cell = src_col + Nx * sr;
      RawSlot raw;
      raw.g0 = __ldg(pg + cell);
      raw.g1 = __ldg(pg + nc + cell);
      raw.g2 = __ldg(pg + 2 * nc + cell);
      const SlotP sl = fold_slot_p<3>(raw, vx, vz, vxz2);
      s_slot[(r * 2) * 32 + lane] = make_float4(sl.lam, sl.c0, sl.c1, sl.c2);
      s_slot[(r * 2 + 1) * 32 + lane] = make_float4(sl.p0, sl.p1, sl.p2, 0.f);
    }
    __syncthreads();
    auto slot_at = [&](int r) {
      const float4 a = s_slot[(r * 2) * 32 + lane], b = s_slot[(r * 2 + 1) * 32 + lane];
      SlotP sl;
      sl.lam = a.x;
      sl.c0 = a.y;
      sl.c1 = a.z;
      sl.c2 = a.w;
      sl.p0 = b.x;
      sl.p1 = b.y;
      sl.p2 = b.z;
      return sl;
    };
    // ---- window: target j at step ky reads staged row w Y + j + (nv - 1 - ky)
    SlotP win[Y];
#pragma unroll
    for (int i = 0; i < Y; ++i) win[i] = slot_at(w * Y + i);
    int qx = x - s_ox[kx];
    if (qx < 0) qx += Nx;
    int qz = z - s_oz[kz];
    if (qz < 0) qz += Nz;
    TS* __restrict__ Fb = F + ((long long)kx + (long long)nv * nv * kz) * nc + qx + (long long)plane * qz;
    float in0[NT][Y], in1[NT][Y], in2[NT][Y];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int j = 0; j < Y; ++j) in0[t][j] = in1[t][j] = in2[t][j] = 0.f;
    for (int kb = nv - 1; kb >= 0; kb -= Y) {
      // this block's f landed (prefetched one block ahead); queue the next
      if (kb - Y >= 0) issue(pr, kb - Y, stage ^ 1);
      else if (pr + 1 < pe) issue(pr + 1, nv - 1, stage ^ 1);
      cp_async_commit();
      cp_async_wait<1>();
#pragma unroll
      for (int jj = 0; jj < Y; ++jj) {
        const int ky = kb - jj;
        const float vy = (g.kmin[1] + ky) * dv;
        const float vy2 = vy * vy;
        float fn[Y];
#pragma unroll
        for (int j = 0; j < Y; ++j) {
          const float f = s_fb[((stage * Y + jj) * Y + j) * NT_ + tid];
          const SlotP& sl = win[(jj + j) % Y];
          const float M = ex2_ftz(fmaf(sl.c2, vy2, fmaf(sl.c1, vy, sl.c0)));
          const float P = fmaf(sl.p2, vy2, fmaf(sl.p1, vy, sl.p0));
          const float fv = fmaf(sl.lam, f, P) + M;
          fn[j] = fv;
          in0[0][j] += fv;
          in1[0][j] = fmaf(fv, vy, in1[0][j]);
          in2[0][j] = fmaf(fv, vy2, in2[0][j]);
          in0[1][j] += M;
          in1[1][j] = fmaf(M, vy, in1[1][j]);
          in2[1][j] = fmaf(M, vy2, in2[1][j]);
        }
        int r = yw - s_oy[ky];
        if (r < 0) r += Ny;
        TS* Fk = Fb + ky * kystep;
#pragma unroll
        for (int j = 0; j < Y; ++j) {
          StreamT<TS>::store(Fk + r * Nx, fn[j]);
          if (++r == Ny) r = 0;
        }
        // slide: the row entering after this step (none after the last)
        const int rin = w * Y + Y + (nv - 1 - ky);
        if (rin < ROWS) win[jj % Y] = slot_at(rin);
      }
      stage ^= 1;
    }
    // the pair's row sums into the split's sums: m = (1, vx, vy, vz, |v|^2/2)
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int j = 0; j < Y; ++j) {
        const float s0 = in0[t][j];
        tot[t][0][j] += s0;
        tot[t][1][j] = fmaf(vx, s0, tot[t][1][j]);
        tot[t][2][j] += in1[t][j];
        tot[t][3][j] = fmaf(vz, s0, tot[t][3][j]);
        tot[t][4][j] += 0.5f * fmaf(vxz2, s0, in2[t][j]);
      }
  }
  cp_async_wait<0>();
  // this split's partial sums: the first part is the new value's sums minus the
  // Maxwellian part's (U_* without its mu''.m part), the second the latter
#pragma unroll
  for (int j = 0; j < Y; ++j) {
    const long long cell = x + (long long)Nx * (yw + j) + (long long)plane * z;
#pragma unroll
    for (int a = 0; a < NM; ++a) {
      p.acc[((long long)split * 2 * NM + a) * nc + cell] = (double)tot[0][a][j] - (double)tot[1][a][j];
      p.acc[((long long)split * 2 * NM + NM + a) * nc + cell] = (double)tot[1][a][j];
    }
  }
}

}  // namespace
}  // namespace dvm
