// dvm_api.cu -- host side of the libdvm C ABI (include/dvm.h): configuration
// checks, the device workspace, the captured CUDA graph of one time step,
// state upload, read-back and checkpoints.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "dvm_internal.cuh"
#include "dvm_learn.cuh"
#include "dvm_readback.cuh"

using namespace dvm;

struct dvm_handle {
  dvm_config cfg;
  Geom g;
  DevPtrs p;
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t cap = nullptr;      // private stream used only for graph capture
  cudaStream_t side = nullptr;     // high-priority stream of the Euler sub-steps
  cudaEvent_t fork = nullptr, join = nullptr;
  bool overlap = true;             // Euler sub-steps concurrent with the kinetic pass
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  void* ws = nullptr;
  bool own_ws = false;
  size_t ws_bytes = 0;
  long long* offs = nullptr;       // small device table for dvm_offsets
  int* pinned_status = nullptr;
  int status = 0;
  std::string err;
  bool state_set = false;
  bool all_free = false;           // every lambda == 1 (tau = inf)
  int launches = 0;
  bool profiling = false;          // bracket each kinetic pass with events
  std::vector<cudaEvent_t> ev0, ev1;
  int nprof = 0;
  // learned regime path
  std::vector<double> lam_host;    // lambda per cell
  std::vector<float> tau_host;     // tau per cell
  dvm_learn_config lcfg{};
  LearnDev L{};
  void* lmem = nullptr;            // one allocation for every learned buffer
  bool params_set = false;
  long long learn_steps = 0;
  long long checks_run = 0;
  cudaGraph_t graph_chk = nullptr; // step with the periodic check
  cudaGraphExec_t exec_chk = nullptr;
  cudaGraph_t graph_multi = nullptr;  // kGraphSteps steps in one graph
  cudaGraphExec_t exec_multi = nullptr;
  float* scratch = nullptr;        // read-back staging (features, labels)
  size_t scratch_bytes = 0;
  dvm::ReadBack rb;                // dvm_moments_async / dvm_moments_wait
};

namespace {

const long long kOffsWidth = kMaxV1;

int fail(dvm_handle* h, int code, const std::string& msg) {
  if (h) {
    if (h->status == 0) h->status = code;
    h->err = msg;
  }
  return code;
}

int cuda_check(dvm_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return 0;
  return fail(h, DVM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t elem_size(int precision) {
  return precision == DVM_F64 ? 8 : (precision == DVM_F32 ? 4 : 2);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace dvm {

// Validate cfg and fill the geometry.  Returns 0 or DVM_ERR_ARG with msg.
int make_geom(const dvm_config* cfg, Geom* g, std::string* msg) {
  if (!cfg) { *msg = "null config"; return DVM_ERR_ARG; }
  const int d = cfg->grid.dim;
  if (d < 1 || d > 3) { *msg = "dim must be 1, 2 or 3"; return DVM_ERR_ARG; }
  memset(g, 0, sizeof(Geom));
  g->d = d;
  g->nm = d + 2;
  g->nc = 1;
  g->nvel = 1;
  for (int i = 0; i < 3; ++i) {
    const int nx = cfg->grid.nx[i], nv = cfg->vel.n[i];
    if (nx < 1 || nv < 1) { *msg = "grid and velocity counts must be >= 1"; return DVM_ERR_ARG; }
    if (i >= d && (nx != 1 || nv != 1)) { *msg = "unused dimensions must have size 1"; return DVM_ERR_ARG; }
    if (nv > kMaxV1) { *msg = "at most 256 velocities per dimension"; return DVM_ERR_ARG; }
    g->nx[i] = nx;
    g->nv[i] = nv;
    g->kmin[i] = i < d ? cfg->vel.kmin[i] : 0;
    g->nc *= nx;
    g->nvel *= nv;
    if (i < d) {
      if (cfg->bc[i][0] != cfg->bc[i][1]) { *msg = "both faces of a dimension need the same boundary rule"; return DVM_ERR_ARG; }
      if (cfg->bc[i][0] != DVM_BC_PERIODIC && cfg->bc[i][0] != DVM_BC_OUTFLOW) { *msg = "unknown boundary rule"; return DVM_ERR_ARG; }
      g->bc[i] = cfg->bc[i][0];
    } else {
      g->bc[i] = DVM_BC_PERIODIC;
    }
  }
  if (!(cfg->grid.dx > 0) || !(cfg->vel.dv > 0) || cfg->vel.shift_den < 1) {
    *msg = "dx, dv must be > 0 and shift_den >= 1";
    return DVM_ERR_ARG;
  }
  if (cfg->scheme < DVM_FKS || cfg->scheme > DVM_FKS_STRANG) { *msg = "unknown scheme"; return DVM_ERR_ARG; }
  if (cfg->precision < DVM_F64 || cfg->precision > DVM_BF16S) { *msg = "unknown precision"; return DVM_ERR_ARG; }
  if (cfg->euler_subcycles < 0 || cfg->max_subcycles < 0) { *msg = "negative sub-step count"; return DVM_ERR_ARG; }
  if (!cfg->tau_field && !(cfg->tau >= 0)) { *msg = "tau must be >= 0"; return DVM_ERR_ARG; }
  g->dx = cfg->grid.dx;
  g->dv = cfg->vel.dv;
  g->p = cfg->vel.shift_den;
  g->w = pow(cfg->vel.dv, d);
  g->dt = cfg->grid.dx / (cfg->vel.shift_den * cfg->vel.dv);
  // Strang-split FKS advances the first-order FKS state (the same moments at
  // every step from equilibrium data) and applies the last half relaxation
  // when f is read out (k_materialize)
  g->strang = cfg->scheme == DVM_FKS_STRANG;
  g->scheme = g->strang ? DVM_FKS : cfg->scheme;
  g->precision = cfg->precision;
  g->forced_sub = cfg->euler_subcycles;
  g->m_cap = cfg->euler_subcycles > 0 ? cfg->euler_subcycles : 0;
  bool outflow = false;
  for (int i = 0; i < d; ++i) outflow |= g->bc[i] == DVM_BC_OUTFLOW;
  g->ghost_mode = outflow ? (d == 1 ? 1 : 2) : 0;
  g->nsplit = kinetic_pass_splits(*g);
  // 3D HOFKS on the windowed pass: one more split for the moments of the
  // transported linear term (dvm_linmom.cu)
  g->lin_slice = g->d == 3 && kinetic_is_windowed(*g) && g->scheme != DVM_FKS ? 1 : 0;
  g->nsplit += g->lin_slice;
  return 0;
}

}  // namespace dvm

namespace {

struct Layout {
  size_t F, ghost, U, lam, W0, W1, Wt, acc, prm, wprm, lin, eqp, gtab, UE, UM, Us, A, small, offs, total;
};

Layout layout(const Geom& g) {
  Layout L;
  const size_t nc = (size_t)g.nc, nv = (size_t)g.nvel, nm = (size_t)g.nm;
  const size_t es = elem_size(g.precision);
  const size_t tc = g.precision == DVM_F64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
  L.F = take(es * nc * nv);
  L.ghost = take(g.ghost_mode == 1 ? es * 2 * nv : (g.ghost_mode == 2 ? es * nc * nv : 0));
  L.U = take(8 * nm * nc);
  L.lam = take(8 * nc);
  L.W0 = take(8 * nm * nc);
  L.W1 = take(8 * nm * nc);
  L.Wt = take(g.scheme == DVM_HOFKS_WENO ? 8 * nm * nc : 0);  // third Runge-Kutta stage
  L.acc = take(8 * (size_t)g.nsplit * 2 * nm * nc);
  L.prm = take(tc * (size_t)prm_rows(g.d) * nc);
  L.wprm = take(g.d >= 2 && g.precision != DVM_F64 ? 4 * 16 * nc : 0);
  L.lin = take(g.lin_slice ? 4 * (size_t)linear_moment_arrays() * nc : 0);
  L.eqp = take(8 * (size_t)prm_rows(g.d) * nc);
  L.gtab = take(g.precision == DVM_F64 ? 8 * nc * (size_t)(1 + g.nv[0] + (g.d > 1 ? g.nv[1] : 0) +
                                                           (g.d > 2 ? g.nv[2] : 0))
                                       : 0);
  L.UE = take(8 * nm * nc);
  L.UM = take(8 * nm * nc);
  L.Us = take(8 * nm * nc);
  L.A = take(8 * kMaxM * kMaxM);
  L.small = take(256);
  L.offs = take(8 * 3 * kOffsWidth);
  L.total = off;
  return L;
}

}  // namespace

namespace dvm {

// (C C^T)^{-1}, C with rows m_k dv^d, by Gauss-Jordan elimination with
// partial pivoting.
int invert_moment_matrix(const Geom& g, double* A) {
  const int nm = g.nm;
  double M[kMaxM][2 * kMaxM];
  memset(M, 0, sizeof M);
  for (long long k = 0; k < g.nvel; ++k) {
    const int kk[3] = {(int)(k % g.nv[0]), (int)((k / g.nv[0]) % g.nv[1]),
                       (int)(k / ((long long)g.nv[0] * g.nv[1]))};
    double m[kMaxM];
    double vv = 0.0;
    m[0] = g.w;
    for (int i = 0; i < g.d; ++i) {
      const double v = (double)(g.kmin[i] + kk[i]) * g.dv;
      m[1 + i] = v * g.w;
      vv += v * v;
    }
    m[g.d + 1] = 0.5 * vv * g.w;
    for (int i = 0; i < nm; ++i)
      for (int j = 0; j < nm; ++j) M[i][j] += m[i] * m[j];
  }
  for (int i = 0; i < nm; ++i) M[i][nm + i] = 1.0;
  for (int col = 0; col < nm; ++col) {
    int piv = col;
    for (int r = col + 1; r < nm; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (!(fabs(M[piv][col]) > 0)) return DVM_ERR_ARG;
    if (piv != col)
      for (int j = 0; j < 2 * nm; ++j) { double t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
    const double inv = 1.0 / M[col][col];
    for (int j = 0; j < 2 * nm; ++j) M[col][j] *= inv;
    for (int r = 0; r < nm; ++r) {
      if (r == col) continue;
      const double f = M[r][col];
      for (int j = 0; j < 2 * nm; ++j) M[r][j] -= f * M[col][j];
    }
  }
  for (int i = 0; i < nm; ++i)
    for (int j = 0; j < nm; ++j) A[i * nm + j] = M[i][nm + j];
  return 0;
}

}  // namespace dvm

namespace {

void bind(dvm_handle* h, char* base, const Layout& L) {
  DevPtrs& p = h->p;
  p.F = base + L.F;
  p.ghost = h->g.ghost_mode ? base + L.ghost : nullptr;
  p.U = (double*)(base + L.U);
  p.lam = (double*)(base + L.lam);
  p.W0 = base + L.W0;
  p.W1 = base + L.W1;
  p.Wt = base + L.Wt;
  p.acc = (double*)(base + L.acc);
  p.prm = base + L.prm;
  p.wprm = (float*)(base + L.wprm);
  p.lin = (float*)(base + L.lin);
  p.eqp = (double*)(base + L.eqp);
  p.gtab = (double*)(base + L.gtab);
  p.UE = (double*)(base + L.UE);
  p.UM = (double*)(base + L.UM);
  p.Us = (double*)(base + L.Us);
  p.A = (double*)(base + L.A);
  char* sm = base + L.small;
  p.alpha = (double*)sm;                              // 3 doubles
  p.alpha_bits = (unsigned long long*)(sm + 32);      // 3
  p.step = (long long*)(sm + 64);
  p.msub = (int*)(sm + 72);
  p.status = (int*)(sm + 76);
  p.counter = (unsigned int*)(sm + 80);
  p.gbar = (unsigned long long*)(sm + 96);            // 1 count
  p.mlast = (int*)(sm + 104);
  p.alpha_prev = (double*)(sm + 112);                 // 3 doubles
  p.aslot = (unsigned long long*)(sm + 144);          // 9
  h->offs = (long long*)(base + L.offs);
}

// Kernels of one time step, in order; e0/e1 (optional) bracket the kinetic pass.
// check: 0 none, 1 the periodic check of seeded cells, 2 the ncheck cells in
// the learned buffer check_cells.
int enqueue_step(dvm_handle* h, cudaStream_t s, cudaEvent_t e0 = nullptr,
                 cudaEvent_t e1 = nullptr, int check = 0, int ncheck = 0) {
  // The Euler sub-steps read only W = (1 - lambda) U^n and write only their
  // own buffers and U_E; the kinetic pass reads only F and the per-cell
  // parameters (nu enters the stored pieces one step later), so the two are
  // independent until the end-of-step kernel, which needs both.  With overlap
  // the Euler kernel runs on a high-priority side stream forked from s.
  const Geom& g = h->g;
  int n = 0;
  if (g.learn) {
    // flags of this step, then the flag-dependent parameters, W and write-back
    cudaMemsetAsync(h->L.mat_count, 0, sizeof(unsigned), s);
    learn_launch_flags(g, h->p, h->L, h->lcfg.mode, h->lcfg.mlp_precision, h->lcfg.thr, s);
    learn_launch_apply(g, h->p, h->L, s);
    n += 2;
    if (kinetic_is_windowed(g)) {
      learn_launch_deep(g, h->L, s);
      n += g.d;
    }
    learn_launch_materialise(g, h->p, h->L, s);
    ++n;
  }
  const bool euler = g.scheme != DVM_FKS && !g.skip_euler;
  // profiled steps stay serial so that the events time the kinetic pass alone.
  // 3D: serial as well -- the kinetic pass holds every SM's registers (3 CTAs
  // of 168-register threads), so nothing runs beside it, and a cooperative
  // Euler grid that finds the SMs taken waits at its grid barrier with part of
  // its CTAs resident, holding shared memory the kinetic pass needs (measured:
  // 64^3 step 7.17 ms serial, 9.78 ms forked)
  const bool fork = euler && h->overlap && !check && !e0 && g.d < 3;
  // 3D windowed HOFKS: the moments of the transported linear term, right
  // before the kinetic pass (inside its events in profiled steps).  On a side
  // stream beside the cooperative Euler grid they delayed its CTAs: 96^3 step
  // 24.4 -> 35.7 ms
  const bool lin = g.lin_slice && kinetic_is_windowed(g);
  if (euler) {
    cudaStream_t es = s;
    if (fork) {
      cudaEventRecord(h->fork, s);
      cudaStreamWaitEvent(h->side, h->fork, 0);
      es = h->side;
    }
    const int rc = cuda_check(h, launch_euler(g, h->p, es), "Euler launch");
    if (rc) return rc;
    ++n;
    if (fork) cudaEventRecord(h->join, h->side);
  }
  if (g.ghost_mode) {
    launch_ghost(g, h->p, s);
    ++n;
  }
  if (check) {
    const int nchk = check == 2 ? ncheck : h->lcfg.check_samples;
    learn_launch_check(g, h->p, h->L, nchk, check == 2, h->lcfg.thr, h->lcfg.veto_radius,
                       h->lcfg.seed, h->lcfg.mode == DVM_LEARN_MLP, s);
    ++n;
  }
  if (e0) cudaEventRecord(e0, s);
  if (lin) n += launch_linear_moments(g, h->p, s);
  n += launch_kinetic_pass(g, h->p, s);
  if (e1) cudaEventRecord(e1, s);
  if (fork) cudaStreamWaitEvent(s, h->join, 0);
  launch_finalize(g, h->p, s);
  ++n;
  h->launches = n;
  return cuda_check(h, cudaGetLastError(), "kernel launch");
}

void drop_graph(dvm_handle* h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->exec_chk) cudaGraphExecDestroy(h->exec_chk);
  if (h->graph_chk) cudaGraphDestroy(h->graph_chk);
  if (h->exec_multi) cudaGraphExecDestroy(h->exec_multi);
  if (h->graph_multi) cudaGraphDestroy(h->graph_multi);
  h->exec = nullptr;
  h->graph = nullptr;
  h->exec_chk = nullptr;
  h->graph_chk = nullptr;
  h->exec_multi = nullptr;
  h->graph_multi = nullptr;
}

// Steps per launch of the multi-step graph: consecutive steps of one call
// run as one graph, without the gap between two graph launches.
constexpr int kGraphSteps = 4;

// Captures one step (check = 0), one step with the periodic check (1), or
// kGraphSteps plain steps (2).
int ensure_graph(dvm_handle* h, int check = 0) {
  cudaGraphExec_t* ex = check == 2 ? &h->exec_multi : (check ? &h->exec_chk : &h->exec);
  cudaGraph_t* gr = check == 2 ? &h->graph_multi : (check ? &h->graph_chk : &h->graph);
  if (!h->use_graph || *ex) return 0;
  int rc = cuda_check(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal),
                      "begin capture");
  if (rc) return rc;
  if (check == 2)
    for (int i = 0; i < kGraphSteps && !rc; ++i) rc = enqueue_step(h, h->cap, nullptr, nullptr, 0);
  else
    rc = enqueue_step(h, h->cap, nullptr, nullptr, check);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
  if (rc) return rc;
  if ((rc = cuda_check(h, e, "end capture"))) return rc;
  *gr = graph;
  return cuda_check(h, cudaGraphInstantiate(ex, graph, 0), "graph instantiate");
}

// A device status word read back to the host: 0, or the handle's sticky error.
int device_status(dvm_handle* h, int st) {
  if (!st) return 0;
  const char* what = st == DVM_ERR_NONFINITE ? "non-finite moments"
                   : st == DVM_ERR_NONPHYSICAL ? "rho <= 0 or theta <= 0 in some cell"
                   : st == DVM_ERR_CFL ? "Euler sub-steps exceed the launch cap"
                   : st == DVM_ERR_TIMEOUT ? "a bounded device wait timed out"
                   : "device error";
  return fail(h, st, what);
}

int sync_status(dvm_handle* h) {
  int rc = cuda_check(h, cudaMemcpyAsync(h->pinned_status, h->p.status, sizeof(int),
                                         cudaMemcpyDeviceToHost, h->stream), "status copy");
  if (rc) return rc;
  if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "stream sync"))) return rc;
  return device_status(h, *h->pinned_status);
}

int ready(dvm_handle* h) {
  if (!h) return DVM_ERR_ARG;
  return h->status;
}

// Shared tail of dvm_set_state_*: U is on the device in h->p.U.
int init_from_moments(dvm_handle* h) {
  const Geom& g = h->g;
  cudaStream_t s = h->stream;
  int rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.status, 0, sizeof(int), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.step, 0, sizeof(long long), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.alpha_bits, 0, 3 * sizeof(unsigned long long) + 0, s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.counter, 0, sizeof(unsigned), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.alpha, 0, 3 * sizeof(double), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.msub, 0, sizeof(int), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.mlast, 0, sizeof(int), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.alpha_prev, 0, 3 * sizeof(double), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.gbar, 0, sizeof(unsigned long long), s), "memset"))) return rc;
  if ((rc = cuda_check(h, cudaMemsetAsync(h->p.aslot, 0, 9 * sizeof(unsigned long long), s), "memset"))) return rc;
  if (h->lmem) {
    // a new state: no cell is flagged (f = E[U] everywhere anyway)
    const size_t nc = (size_t)g.nc;
    if ((rc = cuda_check(h, cudaMemsetAsync(h->L.flag, 0, nc, s), "memset"))) return rc;
    if ((rc = cuda_check(h, cudaMemsetAsync(h->L.flag_prev, 0, nc, s), "memset"))) return rc;
    if ((rc = cuda_check(h, cudaMemsetAsync(h->L.veto, 0, nc, s), "memset"))) return rc;
  }
  launch_cell_params(g, h->p, 0, 1, s);
  launch_init_f(g, h->p, s);
  launch_cell_params(g, h->p, 1, 1, s);
  // alpha, W = (1 - lambda) U^0 and the sub-step count of the first step
  if (g.scheme != DVM_FKS) launch_alpha(g, h->p, s);
  if ((rc = cuda_check(h, cudaGetLastError(), "init launch"))) return rc;
  if ((rc = sync_status(h))) return rc;
  h->state_set = true;
  return 0;
}

// Copy n bytes from a host or device source into device memory.
int upload(dvm_handle* h, void* dst, const void* src, size_t n, int on_device) {
  return cuda_check(h, cudaMemcpyAsync(dst, src, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream), "upload");
}

struct BlobHeader {
  char magic[8];
  int d, nm, precision, scheme;
  int nx[3], nv[3];
  long long step;
  unsigned long long f_bytes, prm_bytes, mom_bytes;
};

}  // namespace

extern "C" {

int dvm_workspace_bytes(const dvm_config* cfg, size_t* bytes) {
  Geom g;
  std::string msg;
  const int rc = make_geom(cfg, &g, &msg);
  if (rc) return rc;
  if (!bytes) return DVM_ERR_ARG;
  *bytes = layout(g).total;
  return 0;
}

int dvm_plan(const dvm_config* cfg, int* kind, int* splits) {
  Geom g;
  std::string msg;
  const int rc = make_geom(cfg, &g, &msg);
  if (rc) return rc;
  if (!kind || !splits) return DVM_ERR_ARG;
  *kind = kinetic_is_windowed(g) ? DVM_KPASS_WINDOW : DVM_KPASS_GENERIC;
  *splits = g.nsplit - g.lin_slice;
  return 0;
}

int dvm_create(const dvm_config* cfg, void* workspace, void* cuda_stream, dvm_handle** out) {
  if (!out) return DVM_ERR_ARG;
  *out = nullptr;
  dvm_handle* h = new dvm_handle();
  std::string msg;
  int rc = make_geom(cfg, &h->g, &msg);
  if (rc) { delete h; return rc; }
  h->cfg = *cfg;
  h->cfg.tau_field = nullptr;
  h->stream = (cudaStream_t)cuda_stream;
  const char* ng = getenv("DVM_NO_GRAPH");
  h->use_graph = !(ng && ng[0] == '1');
  const Layout L = layout(h->g);
  h->ws_bytes = L.total;
  if (workspace) {
    if (((uintptr_t)workspace & 255) != 0) { delete h; return DVM_ERR_ARG; }
    h->ws = workspace;
  } else {
    if (cudaMalloc(&h->ws, L.total) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return DVM_ERR_OOM;
    }
    h->own_ws = true;
  }
  bind(h, (char*)h->ws, L);
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  const char* ov = getenv("DVM_SERIAL_EULER");
  h->overlap = !(ov && ov[0] == '1');
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&h->pinned_status, 64) != cudaSuccess) {
    dvm_destroy(h);
    return DVM_ERR_CUDA;
  }
  double A[kMaxM * kMaxM];
  if (invert_moment_matrix(h->g, A)) { dvm_destroy(h); return DVM_ERR_ARG; }
  kinetic_pass_prepare(h->g);
  std::vector<double> lam((size_t)h->g.nc);
  bool all_free = true;
  for (long long c = 0; c < h->g.nc; ++c) {
    const double tau = cfg->tau_field ? cfg->tau_field[c] : cfg->tau;
    if (!(tau >= 0)) { dvm_destroy(h); return DVM_ERR_ARG; }
    lam[c] = exp(-h->g.dt / tau);
    all_free &= lam[c] == 1.0;
  }
  h->lam_host = lam;
  h->tau_host.resize((size_t)h->g.nc);
  for (long long c = 0; c < h->g.nc; ++c)
    h->tau_host[c] = (float)(cfg->tau_field ? cfg->tau_field[c] : cfg->tau);
  h->all_free = all_free;
  h->g.skip_euler = all_free ? 1 : 0;
  h->g.euler_blocks = euler_blocks(h->g);
  // optional cap of the Euler grid (fewer co-resident blocks leave room on
  // every SM for the concurrent kinetic pass)
  if (const char* eb = getenv("DVM_EULER_BLOCKS")) {
    const int cap = atoi(eb);
    if (cap > 0 && cap < h->g.euler_blocks) h->g.euler_blocks = cap;
  }
  h->g.m_cap = cfg->max_subcycles > 0 ? cfg->max_subcycles : 1000000;
  if (cfg->euler_subcycles > 0 && h->g.m_cap < cfg->euler_subcycles) h->g.m_cap = cfg->euler_subcycles;
  cudaStream_t s = h->stream;
  if (cudaMemsetAsync(h->ws, 0, L.total, s) != cudaSuccess ||
      cudaMemcpyAsync(h->p.A, A, sizeof(double) * h->g.nm * h->g.nm, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(h->p.lam, lam.data(), sizeof(double) * h->g.nc, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    dvm_destroy(h);
    return DVM_ERR_CUDA;
  }
  *out = h;
  return 0;
}

void dvm_destroy(dvm_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  drop_graph(h);
  for (cudaEvent_t e : h->ev0) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev1) cudaEventDestroy(e);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->join) cudaEventDestroy(h->join);
  if (h->pinned_status) cudaFreeHost(h->pinned_status);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->lmem) cudaFree(h->lmem);
  if (h->scratch) cudaFree(h->scratch);
  h->rb.release();
  delete h;
}

int dvm_set_stream(dvm_handle* h, void* cuda_stream) {
  if (!h) return DVM_ERR_ARG;
  h->stream = (cudaStream_t)cuda_stream;
  return 0;
}

const char* dvm_last_error(const dvm_handle* h) {
  return h ? h->err.c_str() : "null handle";
}

int dvm_set_state_moments(dvm_handle* h, const double* U, int on_device) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U) return fail(h, DVM_ERR_ARG, "null moments");
  if ((rc = upload(h, h->p.U, U, sizeof(double) * h->g.nm * h->g.nc, on_device))) return rc;
  return init_from_moments(h);
}

int dvm_set_state_primitive(dvm_handle* h, const double* rho, const double* u, const double* T,
                            int on_device) {
  int rc = ready(h);
  if (rc) return rc;
  if (!rho || !u || !T) return fail(h, DVM_ERR_ARG, "null primitive field");
  const size_t nc = (size_t)h->g.nc;
  double* tmp = nullptr;
  const double *dr = rho, *du = u, *dT = T;
  if (!on_device) {
    // staging in the Euler buffers, which init overwrites anyway
    tmp = (double*)h->p.W0;
    if (3 + h->g.d > 2 * h->g.nm) return fail(h, DVM_ERR_ARG, "staging too small");
    if ((rc = upload(h, tmp, rho, 8 * nc, 0))) return rc;
    if ((rc = upload(h, tmp + nc, u, 8 * nc * h->g.d, 0))) return rc;
    if ((rc = upload(h, tmp + nc * (1 + h->g.d), T, 8 * nc, 0))) return rc;
    dr = tmp;
    du = tmp + nc;
    dT = tmp + nc * (1 + h->g.d);
  }
  launch_prim_to_cons(h->g, dr, du, dT, h->p.U, h->stream);
  if ((rc = cuda_check(h, cudaGetLastError(), "prim launch"))) return rc;
  return init_from_moments(h);
}

int dvm_step_async(dvm_handle* h, int nsteps) {
  int rc = ready(h);
  if (rc) return rc;
  if (!h->state_set) return fail(h, DVM_ERR_STATE, "step before a state was set");
  if (nsteps < 0) return fail(h, DVM_ERR_ARG, "negative step count");
  if (h->profiling) {
    for (int i = 0; i < nsteps; ++i) {
      if (h->nprof >= (int)h->ev0.size()) {
        cudaEvent_t a, b;
        if ((rc = cuda_check(h, cudaEventCreate(&a), "event"))) return rc;
        if ((rc = cuda_check(h, cudaEventCreate(&b), "event"))) return rc;
        h->ev0.push_back(a);
        h->ev1.push_back(b);
      }
      if ((rc = enqueue_step(h, h->stream, h->ev0[h->nprof], h->ev1[h->nprof]))) return rc;
      ++h->nprof;
    }
    return 0;
  }
  if (h->g.learn && h->lcfg.mode == DVM_LEARN_MLP && !h->params_set)
    return fail(h, DVM_ERR_STATE, "network parameters not set");
  for (int i = 0; i < nsteps; ++i) {
    if (!h->g.learn && h->use_graph && nsteps - i >= kGraphSteps) {
      if ((rc = ensure_graph(h, 2))) return rc;
      if ((rc = cuda_check(h, cudaGraphLaunch(h->exec_multi, h->stream), "graph launch"))) return rc;
      i += kGraphSteps - 1;
      continue;
    }
    int check = 0;
    if (h->g.learn) {
      ++h->learn_steps;
      if (h->lcfg.check_every > 0 && h->learn_steps % h->lcfg.check_every == 0) {
        check = 1;
        ++h->checks_run;
      }
    }
    if ((rc = ensure_graph(h, check))) return rc;
    cudaGraphExec_t ex = check ? h->exec_chk : h->exec;
    if (ex) {
      if ((rc = cuda_check(h, cudaGraphLaunch(ex, h->stream), "graph launch"))) return rc;
    } else if ((rc = enqueue_step(h, h->stream, nullptr, nullptr, check))) {
      return rc;
    }
  }
  return 0;
}

int dvm_sync_status(dvm_handle* h) {
  int rc = ready(h);
  if (rc) return rc;
  return sync_status(h);
}

int dvm_step(dvm_handle* h, int nsteps) {
  int rc = dvm_step_async(h, nsteps);
  if (rc) return rc;
  return sync_status(h);
}

int dvm_moments(dvm_handle* h, double* out, int on_device) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out) return fail(h, DVM_ERR_ARG, "null output");
  if ((rc = cuda_check(h, cudaMemcpyAsync(out, h->p.U, sizeof(double) * h->g.nm * h->g.nc,
                                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                          h->stream), "moments copy"))) return rc;
  return cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
}

int dvm_moments_async(dvm_handle* h, double* out, int on_device, long long* ticket) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out || !ticket) return fail(h, DVM_ERR_ARG, "null output or ticket");
  return cuda_check(h, h->rb.issue(h->stream, h->p.U, (long long)h->g.nm * h->g.nc, h->p.status, out,
                                   on_device != 0, ticket), "moments read-back");
}

int dvm_moments_wait(dvm_handle* h, long long ticket) {
  int rc = ready(h);
  if (rc) return rc;
  if (ticket < 0 || ticket >= h->rb.issued) return fail(h, DVM_ERR_ARG, "read-back ticket not issued");
  int st = 0;
  if ((rc = cuda_check(h, h->rb.wait(ticket, &st), "read-back wait"))) return rc;
  return device_status(h, st);
}

int dvm_get_f(dvm_handle* h, double* out, int on_device) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out) return fail(h, DVM_ERR_ARG, "null output");
  const size_t bytes = sizeof(double) * (size_t)h->g.nc * (size_t)h->g.nvel;
  double* dst = out;
  if (!on_device) {
    if ((rc = cuda_check(h, cudaMalloc(&dst, bytes), "f staging"))) return rc;
  }
  launch_materialize(h->g, h->p, dst, h->stream);
  rc = cuda_check(h, cudaGetLastError(), "materialize");
  if (!rc && !on_device)
    rc = cuda_check(h, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream), "f copy");
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  if (!on_device) cudaFree(dst);
  return rc;
}

int dvm_last_parts(dvm_handle* h, double* UE, double* UM, double* Ustar) {
  int rc = ready(h);
  if (rc) return rc;
  if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "sync"))) return rc;
  const size_t b = sizeof(double) * h->g.nm * h->g.nc;
  cudaStream_t s = h->stream;
  if (UE) rc |= cuda_check(h, cudaMemcpyAsync(UE, h->p.UE, b, cudaMemcpyDeviceToHost, s), "copy");
  if (UM) rc |= cuda_check(h, cudaMemcpyAsync(UM, h->p.UM, b, cudaMemcpyDeviceToHost, s), "copy");
  if (Ustar) rc |= cuda_check(h, cudaMemcpyAsync(Ustar, h->p.Us, b, cudaMemcpyDeviceToHost, s), "copy");
  if (rc) return h->status;
  return cuda_check(h, cudaStreamSynchronize(s), "sync");
}

int dvm_info(dvm_handle* h, double* dt, long long* n, int* substeps, double* alpha) {
  int rc = ready(h);
  if (rc) return rc;
  long long step = 0;
  int m = 0;
  double a[3] = {0, 0, 0};
  cudaStream_t s = h->stream;
  rc |= cuda_check(h, cudaMemcpyAsync(&step, h->p.step, sizeof step, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(&m, h->p.msub, sizeof m, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(a, h->p.alpha, sizeof a, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(s), "sync");
  if (rc) return h->status;
  if (dt) *dt = h->g.dt;
  if (n) *n = step;
  if (substeps) *substeps = m;
  if (alpha) memcpy(alpha, a, sizeof a);
  return 0;
}

int dvm_offsets(dvm_handle* h, long long n, long long* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out) return fail(h, DVM_ERR_ARG, "null output");
  int width = 1;
  for (int i = 0; i < h->g.d; ++i) width = h->g.nv[i] > width ? h->g.nv[i] : width;
  launch_offsets(h->g, n, h->offs, width, h->stream);
  if ((rc = cuda_check(h, cudaGetLastError(), "offsets launch"))) return rc;
  if ((rc = cuda_check(h, cudaMemcpyAsync(out, h->offs, sizeof(long long) * h->g.d * width,
                                          cudaMemcpyDeviceToHost, h->stream), "copy"))) return rc;
  return cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
}

int dvm_save(dvm_handle* h, void* buf, size_t* bytes) {
  int rc = ready(h);
  if (rc) return rc;
  if (!bytes) return fail(h, DVM_ERR_ARG, "null size");
  if (!h->state_set) return fail(h, DVM_ERR_STATE, "no state to save");
  if (buf && h->g.learn) {
    // flagged cells hold f = E[U] by definition: write it into their pieces
    learn_launch_flush(h->g, h->p, h->L, h->stream);
    if ((rc = cuda_check(h, cudaGetLastError(), "learned flush"))) return rc;
  }
  const Layout L = layout(h->g);
  BlobHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, "DVMSTAT1", 8);
  hd.d = h->g.d; hd.nm = h->g.nm; hd.precision = h->g.precision; hd.scheme = h->g.scheme;
  for (int i = 0; i < 3; ++i) { hd.nx[i] = h->g.nx[i]; hd.nv[i] = h->g.nv[i]; }
  hd.f_bytes = elem_size(h->g.precision) * (size_t)h->g.nc * (size_t)h->g.nvel;
  hd.prm_bytes = (h->g.precision == DVM_F64 ? 8 : 4) * (size_t)prm_rows(h->g.d) * (size_t)h->g.nc;
  hd.mom_bytes = 8 * (size_t)h->g.nm * (size_t)h->g.nc;
  const size_t total = sizeof hd + hd.f_bytes + hd.prm_bytes + hd.mom_bytes;
  (void)L;
  if (!buf) { *bytes = total; return 0; }
  if (*bytes < total) return fail(h, DVM_ERR_ARG, "checkpoint buffer too small");
  cudaStream_t s = h->stream;
  rc |= cuda_check(h, cudaMemcpyAsync(&hd.step, h->p.step, 8, cudaMemcpyDeviceToHost, s), "copy");
  char* b = (char*)buf + sizeof hd;
  rc |= cuda_check(h, cudaMemcpyAsync(b, h->p.F, hd.f_bytes, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(b + hd.f_bytes, h->p.prm, hd.prm_bytes, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(b + hd.f_bytes + hd.prm_bytes, h->p.U, hd.mom_bytes, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(s), "sync");
  if (rc) return h->status;
  memcpy(buf, &hd, sizeof hd);
  *bytes = total;
  return 0;
}

int dvm_load(dvm_handle* h, const void* buf, size_t bytes) {
  int rc = ready(h);
  if (rc) return rc;
  if (!buf || bytes < sizeof(BlobHeader)) return fail(h, DVM_ERR_ARG, "bad checkpoint");
  BlobHeader hd;
  memcpy(&hd, buf, sizeof hd);
  bool ok = memcmp(hd.magic, "DVMSTAT1", 8) == 0 && hd.d == h->g.d && hd.precision == h->g.precision &&
            hd.scheme == h->g.scheme;
  for (int i = 0; i < 3; ++i) ok &= hd.nx[i] == h->g.nx[i] && hd.nv[i] == h->g.nv[i];
  if (!ok || bytes < sizeof hd + hd.f_bytes + hd.prm_bytes + hd.mom_bytes)
    return fail(h, DVM_ERR_ARG, "checkpoint does not match this configuration");
  cudaStream_t s = h->stream;
  const char* b = (const char*)buf + sizeof hd;
  // the moments first: the cap of Euler sub-steps is derived from them
  rc |= upload(h, h->p.U, b + hd.f_bytes + hd.prm_bytes, hd.mom_bytes, 0);
  if (rc) return h->status;
  if ((rc = init_from_moments(h))) return rc;
  rc |= upload(h, h->p.F, b, hd.f_bytes, 0);
  rc |= upload(h, h->p.prm, b + hd.f_bytes, hd.prm_bytes, 0);
  rc |= cuda_check(h, cudaMemcpyAsync(h->p.step, &hd.step, 8, cudaMemcpyHostToDevice, s), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(s), "sync");
  return rc ? h->status : 0;
}

int dvm_profile_begin(dvm_handle* h) {
  int rc = ready(h);
  if (rc) return rc;
  h->profiling = true;
  h->nprof = 0;
  return 0;
}

int dvm_profile_end(dvm_handle* h, double* kinetic_ms, int* launches) {
  int rc = ready(h);
  if (rc) return rc;
  if (!h->profiling) return fail(h, DVM_ERR_STATE, "profiling was not started");
  h->profiling = false;
  if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "sync"))) return rc;
  double total = 0.0;
  for (int i = 0; i < h->nprof; ++i) {
    float ms = 0.f;
    if ((rc = cuda_check(h, cudaEventElapsedTime(&ms, h->ev0[i], h->ev1[i]), "elapsed"))) return rc;
    total += ms;
  }
  if (kinetic_ms) *kinetic_ms = total;
  if (launches) *launches = h->nprof;
  return 0;
}

int dvm_launches_per_step(dvm_handle* h, int* launches) {
  if (!h || !launches) return DVM_ERR_ARG;
  if (!h->state_set) return fail(h, DVM_ERR_STATE, "no state yet");
  if (h->launches > 0) {  // counted by the last enqueued step
    *launches = h->launches;
    return 0;
  }
  int n = 0;
  if (h->g.scheme != DVM_FKS && !h->g.skip_euler) n += 1;
  if (h->g.ghost_mode) n += 1;
  // (folded parameters or the FP64 Maxwellian factors +) kinetic pass
  n += (kinetic_is_windowed(h->g) || h->g.precision == DVM_F64) ? 2 : 1;
  if (h->g.lin_slice && !h->g.learn) n += 3;  // linear-term moments
  n += 1;                                  // end-of-step kernel
  *launches = n;
  return 0;
}

int dvm_kinetic_kernel(const dvm_handle* h, int* kind) {
  if (!h || !kind) return DVM_ERR_ARG;
  *kind = kinetic_is_windowed(h->g) ? DVM_KPASS_WINDOW : DVM_KPASS_GENERIC;
  return 0;
}

int dvm_kinetic_splits(const dvm_handle* h, int* splits) {
  if (!h || !splits) return DVM_ERR_ARG;
  *splits = h->g.nsplit - h->g.lin_slice;
  return 0;
}

}  // extern "C"

// ------------------------------------------------------------ learned path

namespace {

int learn_alloc(dvm_handle* h) {
  if (h->lmem) return 0;
  const size_t nc = (size_t)h->g.nc;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t off = 0;
  const size_t o_flag = off; off += up(nc);
  const size_t o_prev = off; off += up(nc);
  const size_t o_given = off; off += up(nc);
  const size_t o_veto = off; off += up(nc);
  const size_t o_deep = off; off += up(nc);
  const size_t o_tmp = off; off += up(nc);
  const size_t o_pred = off; off += up(4 * nc);
  const size_t o_tau = off; off += up(4 * nc);
  const size_t o_lw = off; off += up(8 * nc);
  const size_t o_invw = off; off += up(8 * nc);
  const size_t o_P = off; off += up(4 * DVM_MLP_NPARAM);
  const size_t o_Pb = off; off += up(2 * DVM_MLP_NPARAM);
  const size_t o_norm = off; off += up(4 * 2 * DVM_NFEAT);
  const size_t o_list = off; off += up(4 * nc);
  const size_t o_mc = off; off += up(4);
  const size_t o_cnt = off; off += up(8 * kCntN);
  const size_t o_err = off; off += up(8 * 4);
  const size_t o_cc = off; off += up(8 * (size_t)kMaxCheck);
  const size_t o_co = off; off += up(4 * (size_t)kMaxCheck);
  char* b = nullptr;
  if (cudaMalloc((void**)&b, off) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, DVM_ERR_OOM, "learned-path buffers");
  }
  h->lmem = b;
  LearnDev& L = h->L;
  L.flag = (unsigned char*)(b + o_flag);
  L.flag_prev = (unsigned char*)(b + o_prev);
  L.given = (unsigned char*)(b + o_given);
  L.veto = (unsigned char*)(b + o_veto);
  L.deep = (unsigned char*)(b + o_deep);
  L.tmp = (unsigned char*)(b + o_tmp);
  L.pred = (float*)(b + o_pred);
  L.tauf = (float*)(b + o_tau);
  L.lw = (double*)(b + o_lw);
  L.invw = (double*)(b + o_invw);
  L.P = (float*)(b + o_P);
  L.Pb = (__nv_bfloat16*)(b + o_Pb);
  L.norm = (float*)(b + o_norm);
  L.mat_list = (int*)(b + o_list);
  L.mat_count = (unsigned*)(b + o_mc);
  L.cnt = (unsigned long long*)(b + o_cnt);
  L.err = (double*)(b + o_err);
  L.check_cells = (long long*)(b + o_cc);
  L.check_out = (float*)(b + o_co);
  std::vector<double> lw(nc), invw(nc);
  for (size_t c = 0; c < nc; ++c) {
    const double w = 1.0 - h->lam_host[c];
    lw[c] = w > 0.0 ? -log2(w) : INFINITY;
    invw[c] = w > 0.0 ? 1.0 / w : INFINITY;
  }
  cudaStream_t s = h->stream;
  int rc = 0;
  rc |= cuda_check(h, cudaMemsetAsync(b, 0, off, s), "memset");
  rc |= cuda_check(h, cudaMemcpyAsync(L.tauf, h->tau_host.data(), 4 * nc, cudaMemcpyHostToDevice, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(L.lw, lw.data(), 8 * nc, cudaMemcpyHostToDevice, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(L.invw, invw.data(), 8 * nc, cudaMemcpyHostToDevice, s), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(s), "sync");
  return rc ? h->status : 0;
}

int ensure_scratch(dvm_handle* h, size_t bytes) {
  if (h->scratch_bytes >= bytes) return 0;
  if (h->scratch) cudaFree(h->scratch);
  h->scratch = nullptr;
  h->scratch_bytes = 0;
  if (cudaMalloc((void**)&h->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, DVM_ERR_OOM, "read-back staging");
  }
  h->scratch_bytes = bytes;
  return 0;
}

}  // namespace

extern "C" {

int dvm_learn_enable(dvm_handle* h, const dvm_learn_config* cfg) {
  int rc = ready(h);
  if (rc) return rc;
  if (!cfg) return fail(h, DVM_ERR_ARG, "null learned config");
  if (cfg->mode == DVM_LEARN_OFF) {
    if (h->g.learn) {
      if (h->state_set) learn_launch_flush(h->g, h->p, h->L, h->stream);
      if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "learned flush"))) return rc;
      h->g.learn = 0;
      h->p.lflag = nullptr;
      h->p.ldeep = nullptr;
      h->p.linvw = nullptr;
      drop_graph(h);
    }
    return 0;
  }
  if (cfg->mode != DVM_LEARN_GIVEN && cfg->mode != DVM_LEARN_MLP)
    return fail(h, DVM_ERR_ARG, "unknown learned mode");
  if (h->g.scheme == DVM_FKS) return fail(h, DVM_ERR_ARG, "the learned path needs HOFKS");
  if (cfg->mlp_precision != DVM_F32 && cfg->mlp_precision != DVM_BF16S)
    return fail(h, DVM_ERR_ARG, "network precision must be DVM_F32 or DVM_BF16S");
  if (cfg->check_every < 0 || cfg->veto_radius < 0 ||
      (cfg->check_every > 0 && (cfg->check_samples < 1 || cfg->check_samples > kMaxCheck)))
    return fail(h, DVM_ERR_ARG, "bad check settings");
  if ((rc = learn_alloc(h))) return rc;
  float norm[2 * DVM_NFEAT];
  for (int i = 0; i < DVM_NFEAT; ++i) {
    norm[i] = cfg->feat_shift[i];
    norm[DVM_NFEAT + i] = cfg->feat_scale[i];
  }
  if ((rc = cuda_check(h, cudaMemcpyAsync(h->L.norm, norm, sizeof norm, cudaMemcpyHostToDevice,
                                          h->stream), "copy"))) return rc;
  if ((rc = cuda_check(h, cudaStreamSynchronize(h->stream), "sync"))) return rc;
  h->lcfg = *cfg;
  h->g.learn = 1;
  h->p.lflag = h->L.flag;
  h->p.ldeep = h->L.deep;
  h->p.linvw = h->L.invw;
  drop_graph(h);
  return 0;
}

int dvm_learn_set_params(dvm_handle* h, const float* P) {
  int rc = ready(h);
  if (rc) return rc;
  if (!P) return fail(h, DVM_ERR_ARG, "null parameters");
  if (!h->lmem) return fail(h, DVM_ERR_STATE, "learned path not enabled");
  std::vector<__nv_bfloat16> pb(DVM_MLP_NPARAM);
  for (int i = 0; i < DVM_MLP_NPARAM; ++i) pb[i] = __float2bfloat16_rn(P[i]);
  rc |= cuda_check(h, cudaMemcpyAsync(h->L.P, P, 4 * DVM_MLP_NPARAM, cudaMemcpyHostToDevice, h->stream), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(h->L.Pb, pb.data(), 2 * DVM_MLP_NPARAM, cudaMemcpyHostToDevice, h->stream), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  if (rc) return h->status;
  h->params_set = true;
  return 0;
}

int dvm_learn_set_flags(dvm_handle* h, const unsigned char* flags) {
  int rc = ready(h);
  if (rc) return rc;
  if (!flags) return fail(h, DVM_ERR_ARG, "null flags");
  if (!h->lmem) return fail(h, DVM_ERR_STATE, "learned path not enabled");
  rc |= cuda_check(h, cudaMemcpyAsync(h->L.given, flags, (size_t)h->g.nc, cudaMemcpyHostToDevice, h->stream), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  return rc ? h->status : 0;
}

int dvm_learn_flags(dvm_handle* h, unsigned char* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out || !h->lmem) return fail(h, DVM_ERR_ARG, "no learned flags");
  rc |= cuda_check(h, cudaMemcpyAsync(out, h->L.flag, (size_t)h->g.nc, cudaMemcpyDeviceToHost, h->stream), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  return rc ? h->status : 0;
}

int dvm_learn_predictions(dvm_handle* h, float* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out || !h->lmem) return fail(h, DVM_ERR_ARG, "no learned predictions");
  rc |= cuda_check(h, cudaMemcpyAsync(out, h->L.pred, 4 * (size_t)h->g.nc, cudaMemcpyDeviceToHost, h->stream), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  return rc ? h->status : 0;
}

int dvm_learn_get_stats(dvm_handle* h, dvm_learn_stats* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out) return fail(h, DVM_ERR_ARG, "null stats");
  memset(out, 0, sizeof *out);
  if (!h->lmem) return 0;
  unsigned long long cnt[kCntN];
  double err[4];
  const size_t nc = (size_t)h->g.nc;
  std::vector<unsigned char> fl(nc), ve(nc);
  cudaStream_t s = h->stream;
  rc |= cuda_check(h, cudaMemcpyAsync(cnt, h->L.cnt, sizeof cnt, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(err, h->L.err, sizeof err, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(fl.data(), h->L.flag, nc, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaMemcpyAsync(ve.data(), h->L.veto, nc, cudaMemcpyDeviceToHost, s), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(s), "sync");
  if (rc) return h->status;
  long long nf = 0, nv = 0;
  for (size_t c = 0; c < nc; ++c) {
    nf += fl[c] != 0;
    nv += ve[c] != 0;
  }
  out->steps = h->learn_steps;
  out->flagged = nf;
  out->flagged_total = (long long)cnt[kCntFlagged];
  out->materialised = (long long)cnt[kCntMaterialised];
  out->checks = h->checks_run;
  out->checked = (long long)cnt[kCntChecked];
  out->failed = (long long)cnt[kCntFailed];
  out->vetoed = nv;
  out->sum_abs_err = err[0];
  out->max_abs_err = err[1];
  out->max_true = out->checked ? err[2] - 12.0 : 0.0;
  return 0;
}

int dvm_learn_step_checked(dvm_handle* h, int n, const long long* cells, float* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!h->state_set) return fail(h, DVM_ERR_STATE, "step before a state was set");
  if (!h->g.learn) return fail(h, DVM_ERR_STATE, "learned path not enabled");
  if (n < 1 || n > kMaxCheck || !cells || !out) return fail(h, DVM_ERR_ARG, "bad check cells");
  if (h->lcfg.mode == DVM_LEARN_MLP && !h->params_set)
    return fail(h, DVM_ERR_STATE, "network parameters not set");
  for (int i = 0; i < n; ++i)
    if (cells[i] < 0 || cells[i] >= h->g.nc) return fail(h, DVM_ERR_ARG, "check cell out of range");
  cudaStream_t s = h->stream;
  if ((rc = cuda_check(h, cudaMemcpyAsync(h->L.check_cells, cells, 8 * (size_t)n, cudaMemcpyHostToDevice, s), "copy"))) return rc;
  ++h->learn_steps;
  ++h->checks_run;
  if ((rc = enqueue_step(h, s, nullptr, nullptr, 2, n))) return rc;
  if ((rc = cuda_check(h, cudaMemcpyAsync(out, h->L.check_out, 4 * (size_t)n, cudaMemcpyDeviceToHost, s), "copy"))) return rc;
  return sync_status(h);
}

int dvm_features(dvm_handle* h, float* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out) return fail(h, DVM_ERR_ARG, "null output");
  if (!h->state_set) return fail(h, DVM_ERR_STATE, "no state");
  if ((rc = learn_alloc(h))) return rc;
  const size_t bytes = 4 * (size_t)DVM_NFEAT * (size_t)h->g.nc;
  if ((rc = ensure_scratch(h, bytes))) return rc;
  learn_launch_features(h->g, h->p, h->L, h->scratch, h->stream);
  if ((rc = cuda_check(h, cudaGetLastError(), "features launch"))) return rc;
  rc |= cuda_check(h, cudaMemcpyAsync(out, h->scratch, bytes, cudaMemcpyDeviceToHost, h->stream), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  return rc ? h->status : 0;
}

int dvm_noneq(dvm_handle* h, float* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!out) return fail(h, DVM_ERR_ARG, "null output");
  if (!h->state_set) return fail(h, DVM_ERR_STATE, "no state");
  const size_t bytes = 4 * (size_t)h->g.nc;
  if ((rc = ensure_scratch(h, bytes))) return rc;
  learn_launch_noneq(h->g, h->p, h->scratch, h->stream);
  if ((rc = cuda_check(h, cudaGetLastError(), "label launch"))) return rc;
  rc |= cuda_check(h, cudaMemcpyAsync(out, h->scratch, bytes, cudaMemcpyDeviceToHost, h->stream), "copy");
  rc |= cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  return rc ? h->status : 0;
}

}  // extern "C"
