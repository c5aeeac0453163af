// dvm_internal.cuh -- types and device helpers shared by the libdvm
// translation units (never installed, never seen by callers).
//
// Storage of f ("piece storage"): F[k * Nc + q] holds the piecewise-constant
// value of velocity k on piece q.  Pieces never move in memory; after n steps
// the piece q of velocity component k_i sits in cell (q_i + o_i(k_i, n)) mod
// N_i of every dimension i, with o the exact-transport offset of Section 4.2.
// Transport is therefore pure index arithmetic folded into the loads of the
// kinetic pass.
//
// Deferred linear term: the stored value differs from the true f by a term
// that depends only on the cell the piece currently occupies,
//   f = F + omega_s M_k[U_s] + m_k . beta_s     (s = the piece's cell),
// with (omega, beta) = (0, dv^d nu) for HOFKS (the moment-matching correction
// of Eq. minim_full) and (1 - lambda, (1 - lambda) dv^d mu) for FKS (the
// equilibrium part of Eq. relaxdvm).  Applying that term when the piece is
// next read, instead of when it is written, lets one pass over f compute the
// moment sums and the update together: the write no longer has to wait for
// the reduction over all velocities of the cell.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dvm.h"

namespace dvm {

constexpr int kMaxD = 3;
constexpr int kMaxM = 5;      // d + 2
constexpr int kMaxV1 = 256;   // velocities per dimension
constexpr int kMaxNP = 16;

// Per-cell parameter rows (compute type), grouped four rows per 16-byte
// block: row r of cell c at prm[((r / 4) * Nc + c) * 4 + r % 4], so that one
// vector load returns four rows of a cell.  Rows:
//   0            lambda = exp(-dt / tau)
//   1            L = log2(weight * rho / (2 pi theta)^{d/2})
//   2 .. 1+d     u
//   2+d          h = log2(e) / (2 theta)
//   3+d ..       nu' = dv^d nu                      (d+2 rows)
//   3+d+(d+2) .. mu'' = weight * dv^d mu            (d+2 rows)
// (the last row of nu' and of mu'' holds the coefficient of |v|^2, i.e. half
// the energy component, so that m_k . nu = nu0 + nu.v + nu_E |v|^2)
// The Maxwellian of the cell is M_k = exp2(L - h |v_k - u|^2) / weight.
__host__ __device__ inline int prm_rows(int d) { return 4 * ((3 + d + 2 * (d + 2) + 3) / 4); }
__host__ __device__ inline long long prm_at(int row, long long c, long long nc) {
  return ((long long)(row >> 2) * nc + c) * 4 + (row & 3);
}
__host__ __device__ inline int row_lam() { return 0; }
__host__ __device__ inline int row_L() { return 1; }
__host__ __device__ inline int row_u(int i) { return 2 + i; }
__host__ __device__ inline int row_h(int d) { return 2 + d; }
__host__ __device__ inline int row_nu(int d, int i) { return 3 + d + i; }
__host__ __device__ inline int row_mu(int d, int i) { return 3 + d + (d + 2) + i; }

struct Geom {
  int d, nm;
  int nx[3];
  long long nc;
  int nv[3];
  int kmin[3];
  long long nvel;
  double dv, w, dt, dx;
  int p;
  int bc[3];          // DVM_BC_* per dimension
  int scheme;         // DVM_FKS / DVM_HOFKS / DVM_HOFKS_UNLIMITED / DVM_HOFKS_WENO
  int strang;         // FKS with Strang splitting (scheme DVM_FKS_STRANG at dvm_create)
  int precision;      // DVM_F64 / DVM_F32 / DVM_BF16S
  int forced_sub;     // > 0: fixed Euler sub-steps
  int m_cap;          // launch cap of Euler sub-steps
  int nsplit;         // velocity chunks of the kinetic pass (+1: lin_slice)
  int lin_slice;      // 1: the last chunk holds the linear-term moments (dvm_linmom.cu)
  int ghost_mode;     // 0 none, 1 two boundary pieces per velocity (1D), 2 full copy
  int skip_euler;     // every lambda == 1: U_E = 0, no Euler launch
  int euler_blocks;   // grid of the cooperative Euler launch (all co-resident)
  int learn;          // learned regime path on: flagged cells (see dvm_learn.cuh)
};

struct DevPtrs {
  void* F;            // nvel x nc storage
  void* ghost;
  double* U;          // nm x nc
  double* lam;        // nc
  void* W0;           // nm x nc Euler state (ping-pong; FP64 or FP32)
  void* W1;
  void* Wt;           // nm x nc, the WENO solver's Runge-Kutta stage
  double* acc;        // nsplit x 2nm x nc partial moment sums
  void* prm;          // NP x nc, compute type
  float* wprm;        // 16 x nc, the window pass's per-cell parameters (FP32 tiers, d >= 2)
  float* lin;         // linear_moment_arrays() x nc, 1D sums of the linear-term moments (3D)
  double* eqp;        // NP x nc, FP64 parameters of E[U] (initial state only)
  double* gtab;       // FP64 build: (1 + sum_i nv_i) x nc separable Maxwellian factors (k_gauss_tables)
  double* UE;         // nm x nc, last step's U_E (FP64 copy)
  double* UM;         // nm x nc, last step's U_M
  double* Us;         // nm x nc, last step's U_*
  double* A;          // nm x nm, (C C^T)^{-1}
  double* alpha;      // 3, alpha for the coming step
  double* alpha_prev; // 3, alpha used by the last completed step
  int* mlast;         // Euler sub-steps used by the last completed step
  unsigned long long* alpha_bits;  // 3, running max (bit pattern of >= 0 doubles)
  int* msub;          // Euler sub-steps of the current step
  int* status;        // first error code
  long long* step;    // step index n
  unsigned int* counter;  // finished-block counter of the alpha reduction
  unsigned long long* gbar;  // grid barrier of the Euler launch: arrival count
  unsigned long long* aslot;  // 3 x 3: alpha (bit patterns) of Euler sub-steps s, s+1, s+2
  // learned path (null unless Geom::learn): flags of the step, cells whose
  // every source is flagged too, 1 / (1 - lambda)
  const unsigned char* lflag;
  const unsigned char* ldeep;
  const double* linvw;
};

// ---------------------------------------------------------------- helpers

__host__ __device__ inline long long floor_div(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

// Exact-transport offset: round-half-up of k n / p (Section 4.2, pieces
// half-open on the left).
__host__ __device__ inline long long transport_offset(long long k, long long n, long long p) {
  return floor_div(2 * k * n + p, 2 * p);
}

__host__ __device__ inline int wrap(long long x, int n) {
  long long r = x % n;
  return (int)(r < 0 ? r + n : r);
}

__device__ inline void set_status(int* status, int code) { atomicCAS(status, 0, code); }

template <typename T> struct StoreT;
template <> struct StoreT<double> {
  __device__ static double load(const double* p) { return *p; }
  __device__ static void store(double* p, double v) { *p = v; }
};
template <> struct StoreT<float> {
  __device__ static float load(const float* p) { return *p; }
  __device__ static void store(float* p, float v) { *p = v; }
};
template <> struct StoreT<__nv_bfloat16> {
  __device__ static float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ static void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// dvm_api.cu
int make_geom(const dvm_config* cfg, Geom* g, std::string* msg);
int invert_moment_matrix(const Geom& g, double* A);

// ------------------------------------------------------- launch wrappers
// dvm_cells.cu
void launch_prim_to_cons(const Geom& g, const double* rho, const double* u, const double* T,
                         double* U, cudaStream_t s);
// mode: 0 = equilibrium weights (used to build f^0), 1 = parameters of the next step
void launch_cell_params(const Geom& g, const DevPtrs& p, int mode, int initial, cudaStream_t s);
void launch_init_f(const Geom& g, const DevPtrs& p, cudaStream_t s);
void launch_alpha(const Geom& g, const DevPtrs& p, cudaStream_t s);
int euler_blocks(const Geom& g);
cudaError_t launch_euler(const Geom& g, const DevPtrs& p, cudaStream_t s);
void launch_ghost(const Geom& g, const DevPtrs& p, cudaStream_t s);
void launch_finalize(const Geom& g, const DevPtrs& p, cudaStream_t s);
void launch_materialize(const Geom& g, const DevPtrs& p, double* out, cudaStream_t s);
void launch_offsets(const Geom& g, long long n, long long* out, int width, cudaStream_t s);
// dvm_kinetic.cu
int launch_kinetic_pass(const Geom& g, const DevPtrs& p, cudaStream_t s);  // kernels launched
// the windowed pass compiled for a configured shape (dvm_kinetic_shapes.cu):
// launches it (or, with prepare, sets its attributes) and returns true if g is
// one of them (FP32, HOFKS; in 3D without the learned path)
bool launch_window_fixed(const Geom& g, const DevPtrs& p, int splits, cudaStream_t s, bool prepare);
// 3D FP32 HOFKS at a shape the tile kernel is compiled for (dvm_kinetic_shapes.cu)
bool tile3_shape(const Geom& g);
void kinetic_pass_prepare(const Geom& g);
int kinetic_pass_splits(const Geom& g);
bool kinetic_is_windowed(const Geom& g);
// dvm_linmom.cu (3D windowed HOFKS)
int linear_moment_arrays();
int launch_linear_moments(const Geom& g, const DevPtrs& p, cudaStream_t s);  // kernels launched
void linear_moments_prepare(const Geom& g);

}  // namespace dvm
