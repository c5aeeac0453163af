// dvm_kinetic_rows.cu -- the kinetic pass on whole x rows moved by the
// tensor memory accelerator (FP32 storage, 2D and 3D, periodic, p = 1).
//
// The operation is the one of the windowed pass (dvm_kinetic.cu): for every
// target cell and velocity, read the piece covering it (exact transport,
// Section 4.2), add the deferred term of its source cell, relax (FKS: Eq.
// relaxdvm; HOFKS: R then T of Section 4.3.1), accumulate the velocity
// moments (Eq. DM, Eq. UK) and write the piece back in place.
//
// A transport shift maps a whole x row of targets onto a whole x row of
// storage (a rotation by o_x(k, n+1)), so a CTA that owns whole x rows of
// targets reads and writes whole rows of F: every f access of the pass is
// an aligned tensor copy between HBM and shared memory, and the threads
// touch f only in shared memory, at a per-pair rotation of their x index.
// A ring of NST tiles of G*Y*Y rows (G groups of Y target rows, Y velocities
// ky per block) runs NST - 1 blocks ahead of the arithmetic:
//   full[s] (mbarrier) -- the tensor loads of the block landed (tx bytes);
//   done[s] (counter)  -- warps that finished the block and wrote their f
//                         back into the tile.
// The last warp to finish block u stores its rows to HBM, waits until the
// stores have read the tile and loads block u + NST into it.  There is no
// producer warp: the CTA is Nx G threads, a multiple of four warps in the
// usual shapes, so that the register file of every SM sub-partition is used
// evenly.
// Each target row belongs to exactly one CTA per velocity chunk (the tiles
// partition the rows), so a row stored back never overwrites another CTA's
// pieces.  Every wait is bounded: a wait that gives up sets DVM_ERR_TIMEOUT
// and the CTA winds down after its own copies have landed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <stdlib.h>

#include "dvm_internal.cuh"
#include "dvm_window.cuh"

namespace dvm {
namespace {

constexpr int kY = 4;          // target rows per thread, velocities ky per block
constexpr int kStages = 4;     // tiles in the ring
constexpr int kMaxThreads = 512;
constexpr long long kWaitCycles = 1LL << 31;  // ~1 s at 2 GHz

struct RowMaps {
  CUtensorMap rows;  // box {Nx, Y, 1}: Y consecutive rows of one velocity and z plane
  CUtensorMap row;   // box {Nx, 1, 1}: one row (rows that wrap at Ny)
};

struct RowLaunch {
  int G;       // groups of Y target rows per CTA
  int splits;  // velocity chunks across CTAs
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mb_test(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, "
      "p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait of a whole warp for the phase with the given parity: every
// lane waits for it (each lane's wait ends by itself, after ~1 s at most),
// then the warp agrees on the outcome.
__device__ __forceinline__ bool mb_wait(uint64_t* b, unsigned parity) {
  bool done = mb_test(b, parity);
  if (!done) {
    const long long t0 = clock64();
    while (!(done = mb_test(b, parity)) && clock64() - t0 <= kWaitCycles) {
    }
  }
  return __all_sync(0xffffffffu, done);
}
__device__ __forceinline__ void tma_load(float* dst, const CUtensorMap* map, int x, int y, int zk, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4}], [%5];\n" ::"r"(smem_addr(dst)),
      "l"((unsigned long long)(uintptr_t)map), "r"(x), "r"(y), "r"(zk), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store(const CUtensorMap* map, int x, int y, int zk, const float* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                   (unsigned long long)(uintptr_t)map),
               "r"(x), "r"(y), "r"(zk), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Block u of a CTA: velocity pair pb + u / bpb (all compute warps on the same
// pair), first ky = nvy - 1 - (u % bpb) Y.
template <int D, bool HOFKS, bool LEARN>
// 512 threads x 128 registers fill one SM's register file
__global__ void __maxnreg__(128)
    k_kpass_rows(Geom g, DevPtrs p, const __grid_constant__ RowMaps maps, RowLaunch rl) {
  constexpr int Y = kY, NM = D + 2, NA = HOFKS ? 2 * NM : NM, NST = kStages;
  const int Nx = g.nx[0], Ny = g.nx[1], Nz = g.nx[2];
  const int nvx = g.nv[0], nvy = g.nv[1], nvz = g.nv[2];
  const int G = rl.G;
  const int C = Nx * G;  // threads
  const int tid = threadIdx.x;
  const long long nc = g.nc;
  const int plane = Nx * Ny;

  __shared__ __align__(8) uint64_t s_full[NST];
  __shared__ unsigned s_done[NST], s_loads[NST];
  __shared__ int s_ox[kMaxV1], s_oy[kMaxV1], s_oz[kMaxV1];
  __shared__ int s_abort;
  // dynamic: NST tiles [G][Y jj][Y j][Nx] floats, then the FP32 plane sums
  // [NA * Y][C] of the threads
  extern __shared__ __align__(128) float s_dyn[];
  float* s_tile = s_dyn;
  const int tile_floats = G * Y * Y * Nx;
  float* s_mid = s_tile + NST * tile_floats;

  const long long n1 = *p.step + 1;
  for (int t = tid; t < kMaxV1; t += blockDim.x) {
    if (t < nvx) s_ox[t] = wrap((long long)(g.kmin[0] + t) * n1, Nx);
    if (t < nvy) s_oy[t] = wrap((long long)(g.kmin[1] + t) * n1, Ny);
    if (D == 3 && t < nvz) s_oz[t] = wrap((long long)(g.kmin[2] + t) * n1, Nz);
  }
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NST; ++s) {
      mb_init(&s_full[s], 1);
      s_done[s] = 0;
      s_loads[s] = 0;
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int i = 0; i < NA * Y; ++i) s_mid[i * C + tid] = 0.f;

  const int y0 = blockIdx.x * G * Y;  // first target row of the CTA
  const int z = D == 3 ? (int)blockIdx.y : 0;
  const int split = blockIdx.z;
  const int npairs = nvx * (D == 3 ? nvz : 1);
  const int per = npairs / rl.splits;
  const int pb = split * per;
  const int bpb = nvy / Y;
  const int U = per * bpb;

  // this thread's targets: x, rows yt .. yt + Y - 1
  const int x = tid % Nx, grp = tid / Nx;
  const int yt = y0 + grp * Y;
  bool sact[Y];
#pragma unroll
  for (int j = 0; j < Y; ++j) sact[j] = true;
  // learned path: flagged targets keep their pieces (not written back into
  // the tile); a CTA whose targets and all their sources are flagged has
  // U_* = 0 and only writes zero partial sums
  bool skip = false;
  if (LEARN) {
    int all_deep = 1;
#pragma unroll
    for (int j = 0; j < Y; ++j) {
      const long long cell = x + (long long)Nx * (yt + j) + (long long)plane * z;
      sact[j] = !p.lflag[cell];
      all_deep &= p.ldeep[cell] != 0;
    }
    skip = __syncthreads_and(all_deep) != 0;
  } else {
    __syncthreads();
  }
  const unsigned tx_bytes = (unsigned)tile_floats * 4u;
  // tensor copies need 16-byte aligned shared addresses (every tile row is
  // a multiple of 128 bytes from the base)
  if (smem_addr(s_tile) & 15u) {
    if (tid == 0) set_status(p.status, DVM_ERR_ARG);
    return;
  }

  const int warp = tid >> 5, lane = tid & 31;
  // warp 0: the (group, jj) rows of block u, one tensor copy of Y rows or Y
  // single-row copies where the rows wrap at Ny; lane i takes pair i
  auto rows_of = [&](int u, int st, bool store) {
    const int pr = pb + u / bpb;
    const int kb = nvy - 1 - (u % bpb) * Y;
    const int kx = pr % nvx, kz = D == 3 ? pr / nvx : 0;
    int qz = 0;
    if (D == 3) {
      qz = z - s_oz[kz];
      if (qz < 0) qz += Nz;
    }
    float* tile = s_tile + st * tile_floats;
    for (int i = lane; i < G * Y; i += 32) {
      const int gg = i / Y, jj = i % Y;
      const int ky = kb - jj;
      int r = y0 + gg * Y - s_oy[ky];
      if (r < 0) r += Ny;
      const int zk = (kx + nvx * (ky + nvy * kz)) * Nz + qz;
      float* dst = tile + (gg * Y + jj) * Y * Nx;
      if (r + Y <= Ny) {
        if (store) tma_store(&maps.rows, 0, r, zk, dst);
        else tma_load(dst, &maps.rows, 0, r, zk, &s_full[st]);
      } else {
        for (int j = 0; j < Y; ++j) {
          if (store) tma_store(&maps.row, 0, r, zk, dst + j * Nx);
          else tma_load(dst + j * Nx, &maps.row, 0, r, zk, &s_full[st]);
          if (++r == Ny) r = 0;
        }
      }
    }
  };
  auto load_block = [&](int v) {
    if (lane == 0) {
      ++s_loads[v % NST];
      mb_arrive_tx(&s_full[v % NST], tx_bytes);
    }
    __syncwarp();
    rows_of(v, v % NST, false);
  };
  if (warp == 0 && !skip)
    for (int v = 0; v < NST && v < U; ++v) load_block(v);

  // ------------------------------------------------------------ compute
  const float dv = (float)g.dv;
  const float4* __restrict__ pg = (const float4*)p.wprm;  // folded per cell (k_window_fold)
  float lam_c[Y];
  if (!HOFKS) {
#pragma unroll
    for (int j = 0; j < Y; ++j)
      lam_c[j] = __ldg((const float*)p.prm + prm_at(row_lam(), x + Nx * (yt + j) + plane * z, nc));
  }
  int sy_first = (yt - (g.kmin[1] + nvy - 1)) % Ny;
  if (sy_first < 0) sy_first += Ny;
  bool first_plane = true;
  Slot win[Y];
  float in0[NA / NM][Y], in1[NA / NM][Y], in2[NA / NM][Y];
  int rnext = 0, src_base = 0, col = 0;
  float vx = 0.f, vz = 0.f, vxz2 = 0.f;
  bool ok = true;
  for (int u = 0; !skip && u < U; ++u) {
    const int st = u % NST;
    const int pr = pb + u / bpb;
    const int bi = u % bpb;
    const int kb = nvy - 1 - bi * Y;
    if (bi == 0) {
      // a new velocity pair: its vx, vz, the rotation of this thread's
      // column in the stored rows, and the first Y sources of the window
      const int kx = pr % nvx, kz = D == 3 ? pr / nvx : 0;
      const int kxg = g.kmin[0] + kx, kzg = D == 3 ? g.kmin[2] + kz : 0;
      vx = kxg * dv;
      vz = kzg * dv;
      vxz2 = fmaf(vx, vx, vz * vz);
      int sx = (x - kxg) % Nx;
      if (sx < 0) sx += Nx;
      int sz = 0;
      if (D == 3) {
        sz = (z - kzg) % Nz;
        if (sz < 0) sz += Nz;
      }
      src_base = sx + plane * sz;
      col = x - s_ox[kx];
      if (col < 0) col += Nx;
      rnext = sy_first;
#pragma unroll
      for (int i = 0; i < Y; ++i) {
        win[i] = load_slot<D>(pg, nc, src_base + Nx * rnext, vx, vz, vxz2);
        if (++rnext == Ny) rnext = 0;
      }
#pragma unroll
      for (int t = 0; t < NA / NM; ++t)
#pragma unroll
        for (int j = 0; j < Y; ++j) in0[t][j] = in1[t][j] = in2[t][j] = 0.f;
    }
    if (!mb_wait(&s_full[st], (unsigned)((u / NST) & 1))) {
      ok = false;
      break;
    }
    float* tile = s_tile + st * tile_floats + grp * Y * Y * Nx + col;
#pragma unroll
    for (int jj = 0; jj < Y; ++jj) {
      const int ky = kb - jj;
      // the source row entering the window after this step (loaded and
      // folded after the last step of a pair too, unused)
      RawSlot raw;
      const int src_next = src_base + Nx * rnext;
      raw.g0 = __ldg(pg + src_next);
      raw.g1 = __ldg(pg + nc + src_next);
      const float vy = (g.kmin[1] + ky) * dv;
      const float vy2 = vy * vy;
      float* trow = tile + jj * Y * Nx;
#pragma unroll
      for (int j = 0; j < Y; ++j) {
        const Slot& sl = win[(jj + j) % Y];
        const float f = trow[j * Nx];
        const float M = ex2_ftz(fmaf(sl.c2, vy2, fmaf(sl.c1, vy, sl.c0)));
        const float lm = fmaf(sl.b2, vy2, fmaf(sl.b1, vy, sl.b0));
        float fn;
        if (HOFKS) {
          const float a = fmaf(sl.lam, f, fmaf(sl.a2, vy2, fmaf(sl.a1, vy, sl.a0)));
          const float b = M + lm;  // T((1 - lambda) E^n)
          fn = a + b;              // a = T(lambda f^n)
          in0[0][j] += a;
          in1[0][j] = fmaf(a, vy, in1[0][j]);
          in2[0][j] = fmaf(a, vy2, in2[0][j]);
          in0[NA / NM - 1][j] += b;
          in1[NA / NM - 1][j] = fmaf(b, vy, in1[NA / NM - 1][j]);
          in2[NA / NM - 1][j] = fmaf(b, vy2, in2[NA / NM - 1][j]);
        } else {
          const float fs = f + M + lm;  // transported f
          fn = lam_c[j] * fs;           // its lambda part; the rest is deferred
          in0[0][j] += fs;
          in1[0][j] = fmaf(fs, vy, in1[0][j]);
          in2[0][j] = fmaf(fs, vy2, in2[0][j]);
        }
        if (!LEARN || sact[j]) trow[j * Nx] = fn;
      }
      raw.g2 = __ldg(pg + 2 * nc + src_next);
      raw.g3 = __ldg(pg + 3 * nc + src_next);
      win[jj % Y] = fold_slot<D>(raw, vx, vz, vxz2);
      if (++rnext == Ny) rnext = 0;
    }
    // this warp is done with the tile; the last one stores the block and
    // loads block u + NST into the tile once the stores have read it
    __syncwarp();
    unsigned before = 0;
    if (lane == 0) {
      __threadfence_block();
      before = atomicAdd(&s_done[st], 1u);
      __threadfence_block();
    }
    before = __shfl_sync(0xffffffffu, before, 0);
    if (before == (unsigned)(C / 32) - 1) {
      fence_proxy_async();
      rows_of(u, st, true);
      bulk_commit();
      bulk_wait_read0();
      __syncwarp();
      if (lane == 0) s_done[st] = 0;
      if (u + NST < U) load_block(u + NST);
    }
    if (bi == bpb - 1) {
      // fold the row sums into the plane sums: m = (1, vx, vy, [vz], |v|^2/2)
#pragma unroll
      for (int t = 0; t < NA / NM; ++t) {
        const int o = t * NM;
#pragma unroll
        for (int j = 0; j < Y; ++j) {
          const float s0 = in0[t][j];
          float* m = s_mid + tid;
          m[((o + 0) * Y + j) * C] += s0;
          m[((o + 1) * Y + j) * C] = fmaf(vx, s0, m[((o + 1) * Y + j) * C]);
          m[((o + 2) * Y + j) * C] += in1[t][j];
          if (D == 3) m[((o + 3) * Y + j) * C] = fmaf(vz, s0, m[((o + 3) * Y + j) * C]);
          m[((o + D + 1) * Y + j) * C] += 0.5f * fmaf(vxz2, s0, in2[t][j]);
        }
      }
      // a finished kz plane (or the chunk's last pair): FP32 plane sums
      // into this thread's FP64 partial sums in HBM
      if ((pr + 1) % nvx == 0 || pr + 1 == pb + per) {
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int j = 0; j < Y; ++j) {
            const long long cell = x + (long long)Nx * (yt + j) + (long long)plane * z;
            double* dst = p.acc + ((long long)split * 2 * NM + a) * nc + cell;
            float* m = s_mid + (a * Y + j) * C + tid;
            *dst = (first_plane ? 0.0 : *dst) + (double)*m;
            *m = 0.f;
          }
        first_plane = false;
      }
    }
    if (__any_sync(0xffffffffu, *(volatile int*)&s_abort != 0)) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    set_status(p.status, DVM_ERR_TIMEOUT);
    s_abort = 1;
    // loads still in flight land before the CTA's shared memory goes away
    // (the latest load of every tile; its phase parity from the count)
    if (warp == 0)
      for (int t = 0; t < NST; ++t) {
        const unsigned nl = *(volatile unsigned*)&s_loads[t];
        if (nl) mb_wait(&s_full[t], (nl - 1) & 1u);
      }
  }
  bulk_wait0();  // this warp's stores
  if (!ok) return;
  if (skip || U == 0) {
    for (int a = 0; a < NA; ++a)
#pragma unroll
      for (int j = 0; j < Y; ++j) {
        const long long cell = x + (long long)Nx * (yt + j) + (long long)plane * z;
        p.acc[((long long)split * 2 * NM + a) * nc + cell] = 0.0;
      }
  }
}

size_t rows_smem(const Geom& g, int G) {
  const bool ho = g.scheme != DVM_FKS;
  const size_t na = (size_t)(ho ? 2 : 1) * (g.d + 2);
  return 128 + (size_t)kStages * G * kY * kY * g.nx[0] * sizeof(float) +
         na * kY * (size_t)g.nx[0] * G * sizeof(float);
}

// CTA shape: G groups of Y target rows, G the largest with Nx G <= 512
// threads, Ny divisible by G Y (the tiles partition the rows) and the
// tiles and plane sums within the shared memory of an SM.
int rows_groups(const Geom& g) {
  int best = 0;
  for (int G = 1; G * g.nx[0] <= kMaxThreads && G <= 16; ++G)
    if (g.nx[1] % (G * kY) == 0 && rows_smem(g, G) <= 227 * 1024) best = G;
  return best;
}

// Velocity chunks: the smallest divisor (of the kz planes in 3D, of the kx
// values in 2D) that gives two waves of one CTA per SM, at most 16.
int rows_splits(const Geom& g, int G) {
  const long long tiles = (long long)(g.nx[1] / (G * kY)) * g.nx[2];
  const long long want = 152LL * 2;
  const int units = g.d == 3 ? g.nv[2] : g.nv[0];
  int sp = 1;
  for (int c = 1; c <= 16 && c <= units; ++c) {
    if (units % c) continue;
    sp = c;
    if (tiles * c >= want) break;
  }
  return sp;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    else
      cudaGetLastError();  // no driver here: the row pass is not offered
  }
  return fn;
}

// F (FP32, index k nc + z Nx Ny + y Nx + x) as a rank-3 tensor {Nx, Ny,
// Nz nvel}: the x row of storage row y, plane z, velocity k is at (0, y, k Nz + z).
bool encode_maps(const Geom& g, void* F, RowMaps* m) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx[0], (cuuint64_t)g.nx[1], (cuuint64_t)g.nx[2] * (cuuint64_t)g.nvel};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx[0] * 4, (cuuint64_t)g.nx[0] * g.nx[1] * 4};
  const cuuint32_t box_rows[3] = {(cuuint32_t)g.nx[0], (cuuint32_t)kY, 1};
  const cuuint32_t box_row[3] = {(cuuint32_t)g.nx[0], 1, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  if (enc(&m->rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, F, dims, strides, box_rows, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  return enc(&m->row, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, F, dims, strides, box_row, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int D, bool HO, bool LE>
void set_rows_smem(size_t bytes) {
  cudaFuncSetAttribute(k_kpass_rows<D, HO, LE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Opt-in (DVM_ROWS_PASS=1): on GB300 the windowed pass is faster.  With
// every warp of a CTA on the same velocity pair and most of the shared memory
// holding the tiles, the per-source parameters miss L1 (9 % hits at 32^3 x
// 24^3, 2.6x the f traffic re-read from L2), while the windowed pass's warps
// on neighbouring pairs share their lines.
bool kinetic_rows_allowed(const Geom& g) {
  const char* e = getenv("DVM_ROWS_PASS");
  if (!(e && e[0] == '1')) return false;
  if (g.precision != DVM_F32 || g.d < 2 || g.p != 1) return false;
  for (int i = 0; i < g.d; ++i)
    if (g.bc[i] != DVM_BC_PERIODIC) return false;
  // a tensor-copy box is at most 256 elements wide
  if (g.nx[0] % 32 || g.nx[0] > 256 || g.nv[1] % kY || g.nx[1] < kY) return false;
  if (g.nc >= (1LL << 31) || (long long)g.nx[2] * g.nvel >= (1LL << 31)) return false;
  return rows_groups(g) > 0 && encode_fn() != nullptr;
}

int kinetic_rows_splits(const Geom& g) { return rows_splits(g, rows_groups(g)); }

void kinetic_rows_prepare(const Geom& g) {
  const size_t sm = rows_smem(g, rows_groups(g));
  set_rows_smem<2, true, false>(sm);
  set_rows_smem<2, true, true>(sm);
  set_rows_smem<2, false, false>(sm);
  set_rows_smem<2, false, true>(sm);
  set_rows_smem<3, true, false>(sm);
  set_rows_smem<3, true, true>(sm);
  set_rows_smem<3, false, false>(sm);
  set_rows_smem<3, false, true>(sm);
}

cudaError_t launch_kinetic_rows(const Geom& g, const DevPtrs& p, cudaStream_t s) {
  RowMaps maps;
  if (!encode_maps(g, p.F, &maps)) return cudaErrorInvalidValue;
  RowLaunch rl;
  rl.G = rows_groups(g);
  rl.splits = rows_splits(g, rl.G);
  const size_t sm = rows_smem(g, rl.G);
  const dim3 grid((unsigned)(g.nx[1] / (rl.G * kY)), (unsigned)g.nx[2], (unsigned)rl.splits);
  const unsigned threads = (unsigned)(g.nx[0] * rl.G);
  const bool ho = g.scheme != DVM_FKS;
#define DVM_ROWS(DD, HO, LE) k_kpass_rows<DD, HO, LE><<<grid, threads, sm, s>>>(g, p, maps, rl)
  if (g.d == 2) {
    if (ho) { if (g.learn) DVM_ROWS(2, true, true); else DVM_ROWS(2, true, false); }
    else { if (g.learn) DVM_ROWS(2, false, true); else DVM_ROWS(2, false, false); }
  } else {
    if (ho) { if (g.learn) DVM_ROWS(3, true, true); else DVM_ROWS(3, true, false); }
    else { if (g.learn) DVM_ROWS(3, false, true); else DVM_ROWS(3, false, false); }
  }
#undef DVM_ROWS
  return cudaGetLastError();
}

}  // namespace dvm
