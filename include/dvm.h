/*
 * dvm.h -- C ABI of libdvm, the GB300 (sm_103a) implementation of the fast
 * kinetic schemes FKS and HOFKS for the discrete-velocity BGK equation of
 * Dimarco & Loubere, "Towards an ultra efficient kinetic scheme, Part II: the
 * high order case" (arXiv:1212.0204).
 *
 * Model (Sections 2-3): f(x, v, t) on a uniform Cartesian cell grid in d = 1..3
 * space dimensions and a tensor grid of N_v discrete velocities v_k = k dv in
 * the same number of velocity dimensions, relaxing towards the conservative
 * discrete Maxwellian E[U] with relaxation time tau.
 *
 * Conventions shared by every entry point:
 *  - Status: every function returns an int; 0 (DVM_OK) on success, a negative
 *    dvm_status otherwise.  Errors are sticky per handle: after a failure the
 *    handle rejects further work with the same code; dvm_last_error() gives a
 *    one-line message.
 *  - Streams: all device work is enqueued on the CUDA stream given to
 *    dvm_create (or dvm_set_stream); NULL means the legacy default stream.
 *    Calls that return data to the host synchronise that stream.
 *  - Pointers: "device" pointers are CUDA device addresses, "host" pointers are
 *    ordinary (pageable or pinned) host memory; an on_device flag says which.
 *    The library never frees a caller buffer.
 *  - Cell order: c = x + nx[0] * (y + nx[1] * z), x fastest.
 *    Velocity order: k = kx + nv[0] * (ky + nv[1] * kz), kx fastest, with
 *    v_i = (kmin[i] + k_i) * dv.
 *  - Moments U (Eq. DM): structure of arrays, FP64, (d+2) rows of N_c values:
 *    rho, rho u_1 .. rho u_d, E with E = rho |u|^2 / 2 + d rho theta / 2
 *    (Eq. E, gas constant R = 1 so theta = T).
 */
#ifndef DVM_H
#define DVM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DVM_OK = 0,
  DVM_ERR_ARG = -1,         /* invalid argument or configuration */
  DVM_ERR_OOM = -2,         /* device allocation failed or workspace too small */
  DVM_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  DVM_ERR_NONFINITE = -4,   /* a moment became NaN or infinite */
  DVM_ERR_NONPHYSICAL = -5, /* rho <= 0 or theta <= 0 in some cell */
  DVM_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up */
  DVM_ERR_STATE = -7,       /* call out of order (e.g. step before a state is set) */
  DVM_ERR_CFL = -8,         /* Euler sub-steps needed exceed max_subcycles */
  DVM_ERR_TOO_LARGE = -9    /* problem larger than the fixed scratch of
                               dvm_equilibrium_noalloc */
} dvm_status;

/* Size of the fixed device scratch array used by dvm_equilibrium_noalloc. */
#define DVM_NOALLOC_SCRATCH_BYTES (8u << 20)
/* Bytes at the start of that array before the per-cell parameters (status
 * word and (C C^T)^{-1}). */
#define DVM_NOALLOC_HEADER_BYTES 512u

typedef enum { DVM_BC_PERIODIC = 0, DVM_BC_OUTFLOW = 1 } dvm_bc;
/* DVM_HOFKS_WENO: HOFKS with the WENO5 Euler solver of Section 4.3.3 (finite-
 * difference WENO5 on the split fluxes (F +- alpha U)/2, three-stage SSP
 * Runge-Kutta per Euler sub-step) in place of MUSCL; single problems only. */
/* DVM_FKS_STRANG: FKS with the Strang splitting Section 4.2 names as the more
 * accurate alternative (relaxation over dt/2, exact transport, relaxation
 * over dt/2 each step).  From the equilibrium data dvm_set_state_* builds,
 * its moments after every step equal those of DVM_FKS, and its f is the FKS
 * state relaxed by half a step less: f - E[U] = (f_FKS - E[U]) / lambda_h,
 * lambda_h = exp(-dt/(2 tau)); the library advances the FKS state and
 * applies that relation where f is read (dvm_get_f).  Single problems only. */
typedef enum { DVM_FKS = 0, DVM_HOFKS = 1, DVM_HOFKS_UNLIMITED = 2, DVM_HOFKS_WENO = 3,
               DVM_FKS_STRANG = 4 } dvm_scheme;
typedef enum { DVM_F64 = 0, DVM_F32 = 1, DVM_BF16S = 2 } dvm_precision;

/* Spatial grid (Section 4): cell centres x0 + (j + 1/2) dx per dimension. */
typedef struct {
  int dim;       /* d = 1, 2 or 3 */
  int nx[3];     /* cells per dimension; entries beyond dim must be 1 */
  double x0[3];  /* lower corner of the domain */
  double dx;     /* uniform cell size */
} dvm_grid;

/* Velocity grid (Section 3) with a = 0: v_i = k_i dv, k_i = kmin_i ..
 * kmin_i + n_i - 1.  The time step is dt = dx / (shift_den * dv), so that a
 * piece moves k_i / shift_den cells per step (exact transport, Section 4.2);
 * shift_den = 1 gives integer shifts. */
typedef struct {
  int n[3];       /* velocities per dimension; entries beyond dim must be 1 */
  int kmin[3];
  double dv;
  int shift_den;  /* p >= 1 */
} dvm_vset;

typedef struct {
  dvm_grid grid;
  dvm_vset vel;
  double tau;               /* uniform relaxation time; INFINITY = free transport */
  const double* tau_field;  /* NULL, or N_c host values overriding tau */
  dvm_bc bc[3][2];          /* per dimension and face; both faces of a
                               dimension must agree */
  int scheme;               /* dvm_scheme; DVM_HOFKS is the paper's scheme */
  int precision;            /* dvm_precision: storage type of f */
  int euler_subcycles;      /* 0: MUSCL sub-steps by Eq. Time2, each with the
                               alpha of its own initial state, the last one
                               ending at dt; > 0: that many equal sub-steps */
  int max_subcycles;        /* cap on sub-steps per kinetic step, exceeding it
                               sets DVM_ERR_CFL; 0 = 10^6 */
} dvm_config;

typedef struct dvm_handle dvm_handle;

/* Bytes of device workspace dvm_create needs for cfg (f, moments, Euler
 * buffers, per-cell parameters, partial sums).  Returns DVM_ERR_ARG for an
 * invalid configuration. */
int dvm_workspace_bytes(const dvm_config* cfg, size_t* bytes);

/* Create a solver.  workspace: NULL (the library allocates with cudaMalloc
 * and frees in dvm_destroy) or a device buffer of at least
 * dvm_workspace_bytes bytes, 256-byte aligned, owned by the caller and kept
 * alive until dvm_destroy.  cuda_stream: a cudaStream_t or NULL.  The step
 * of one time level is captured once into a CUDA graph here.  The state is
 * empty until dvm_set_state_* is called.  tau_field is copied. */
int dvm_create(const dvm_config* cfg, void* workspace, void* cuda_stream,
               dvm_handle** out);
void dvm_destroy(dvm_handle* h);
int dvm_set_stream(dvm_handle* h, void* cuda_stream);
const char* dvm_last_error(const dvm_handle* h);

/* Initial state in thermodynamic equilibrium: f^0 = E[U^0] (Eq. minimMax,
 * the projection of Eq. minim1 applied to the pointwise Maxwellian,
 * Section 4.2 "first time step").  U: (d+2) x N_c FP64 moments, host or
 * device.  Resets the step counter to 0.  DVM_ERR_NONPHYSICAL if some cell
 * has rho <= 0 or theta <= 0. */
int dvm_set_state_moments(dvm_handle* h, const double* U, int on_device);

/* Same from primitive fields (Eqs. Mo, E): rho[N_c], u[d x N_c], T[N_c]. */
int dvm_set_state_primitive(dvm_handle* h, const double* rho, const double* u,
                            const double* T, int on_device);

/* Advance nsteps time levels (FKS: Section 4.2, transport then relaxation;
 * HOFKS: Section 4.3.1, relaxation, transport, U_M replaced by the MUSCL
 * Euler moments U_E of Section 4.3.2 and the equilibrium part matched to
 * U_E by Eq. minim_full).  Enqueues the captured graph nsteps times, then
 * synchronises the stream and returns the device status word (first error
 * wins: DVM_ERR_NONFINITE, DVM_ERR_NONPHYSICAL, DVM_ERR_CFL). */
int dvm_step(dvm_handle* h, int nsteps);

/* As dvm_step without the final synchronisation; the status is read later
 * by dvm_sync_status. */
int dvm_step_async(dvm_handle* h, int nsteps);
int dvm_sync_status(dvm_handle* h);

/* Moments U^n at t = n dt (for HOFKS the hybrid moments U_H of Eq. mom):
 * (d+2) x N_c FP64 into the caller's buffer (host or device). */
int dvm_moments(dvm_handle* h, double* out, int on_device);

/* Pipelined read-back of the same moments after every step enqueued so far,
 * for a caller that reads each step's result while later steps run.  The
 * moments and the status word are copied on the device in stream order into
 * one of two snapshot slots, and from there into `out` ((d+2) x N_c FP64,
 * host -- pinned for an asynchronous copy -- or device; caller-owned, left
 * untouched by the library after dvm_moments_wait returns, and not to be read
 * or freed before) on a private copy stream.  At most two read-backs are in
 * flight: the stream of the steps waits (on the device) until a slot's
 * previous copy has left it before reusing it.  *ticket (0, 1, 2, ... per
 * handle) names the read-back for dvm_moments_wait.  The first call allocates
 * the two slots (2 (d+2) N_c doubles) and must come before any capture of
 * the handle's stream.  Errors: DVM_ERR_ARG (null out or ticket), a CUDA
 * failure (DVM_ERR_CUDA). */
int dvm_moments_async(dvm_handle* h, double* out, int on_device, long long* ticket);

/* Blocks until read-back `ticket` is in its output buffer (copies complete
 * in ticket order), then returns the device status word as that ticket's
 * snapshot found it: DVM_OK or the error code, which also becomes the
 * handle's sticky error like dvm_step's.  The statuses of the last 64
 * tickets are kept; an older ticket waits for the newest read-back and
 * reports its status (the device status is sticky, so it holds at least the
 * older ticket's error).  DVM_ERR_ARG for a ticket not issued. */
int dvm_moments_wait(dvm_handle* h, long long ticket);

/* f^n at the cell centres, N_v x N_c FP64 (velocity-major), materialised
 * from the piece storage (the library never moves f; see dvm_offsets). */
int dvm_get_f(dvm_handle* h, double* out, int on_device);

/* U_E, U_M and U_* of the last HOFKS step (Eqs. UK and mom), each
 * (d+2) x N_c FP64 host arrays; any pointer may be NULL. */
int dvm_last_parts(dvm_handle* h, double* UE, double* UM, double* Ustar);

/* dt, step index n, MUSCL sub-steps and alpha (per direction) of the last
 * step.  Synchronises the stream. */
int dvm_info(dvm_handle* h, double* dt, long long* n, int* substeps,
             double* alpha);

/* Exact-transport offsets o_i(k_i, n) = floor((2 k_i n + p) / (2 p)), the
 * number of cells the piece of velocity component k_i has moved after n
 * steps (pieces half-open on the left), computed by the same device code the
 * kinetic pass uses.  out: host int64 array of d x max_i(n_i) entries, row i
 * holding dimension i. */
int dvm_offsets(dvm_handle* h, long long n, long long* out);

/* Checkpoint: the full state (step index, piece storage of f, moments and
 * per-cell parameters) as an opaque host blob.  With buf == NULL, *bytes
 * receives the size.  dvm_load restores it into a handle created with the
 * same configuration; the run then continues bit for bit. */
int dvm_save(dvm_handle* h, void* buf, size_t* bytes);
int dvm_load(dvm_handle* h, const void* buf, size_t bytes);

/* Kernel launches enqueued by one time step (the captured graph's nodes). */
int dvm_launches_per_step(dvm_handle* h, int* launches);

/* Which kinetic-pass kernel the handle's steps run (chosen at dvm_create
 * from the grid, precision and boundaries): DVM_KPASS_GENERIC (one thread
 * per cell, any configuration) or DVM_KPASS_WINDOW (FP32/BF16 storage,
 * periodic 2D/3D, p = 1: windows of source rows that slide along the
 * velocity; at the configured 3D FP32 shapes the CTA shares them). */
enum { DVM_KPASS_GENERIC = 0, DVM_KPASS_WINDOW = 1 };
int dvm_kinetic_kernel(const dvm_handle* h, int* kind);

/* Velocity chunks of the kinetic pass (chosen at dvm_create from the grid and
 * the SM count): the velocity loop of every target cell is split over this
 * many CTAs, each writing its own FP64 partial moment sums, which the
 * end-of-step kernel adds (Eq. DM summed in parts).  1 = no split. */
int dvm_kinetic_splits(const dvm_handle* h, int* splits);

/* The kinetic-pass plan dvm_create would choose for cfg, without creating
 * anything or touching a GPU: the kernel kind (as dvm_kinetic_kernel) and
 * its velocity chunks (as dvm_kinetic_splits), for the SM count of the
 * current device, or 152 SMs (GB300) when no device is visible.  The split
 * count follows the fill of the last wave of CTAs (Section 4.2's pass over
 * the velocities, summed in parts).  Host only; DVM_ERR_ARG for an invalid
 * configuration or a NULL output. */
int dvm_plan(const dvm_config* cfg, int* kind, int* splits);

/* Kinetic-pass timing.  Between dvm_profile_begin and dvm_profile_end the
 * steps are enqueued launch by launch (not through the graph) with a pair of
 * CUDA events recorded on the handle's stream around every kinetic-pass
 * launch.  dvm_profile_end synchronises the stream and returns the summed
 * kinetic-pass time in milliseconds and the number of launches timed. */
int dvm_profile_begin(dvm_handle* h);
int dvm_profile_end(dvm_handle* h, double* kinetic_ms, int* launches);

/* ----------------------------------------------------------------------
 * Batched 1D-1V and 2D-2V cases.  Many independent problems (each with its
 * own dimension, grid, velocity set, tau, p and boundary rule; all with the
 * same scheme and precision, scalar tau; a 1D tube has N_x <= 4096 cells, a
 * 2D case is periodic in both dimensions with at most 2^20 cells) advance
 * together: one time step of the batch is three kernel launches for all
 * cases, captured into one CUDA graph (Euler sub-steps, one CTA per case; one
 * persistent kinetic pass over a work queue of (case, cell tile, velocity
 * chunk) items ordered by cost; end-of-step update).  The scheme is the one
 * of dvm_step (Sections 4.2 and 4.3; Section 4.2 is dimension-generic).
 * Packed layout of batch moments: R rows (R = dvm_batch_moment_rows: 3 if
 * every case is 1D, else 4) of N_total cells each, FP64; case i's cells
 * (x fastest) at [c_i, c_i + N_cells,i), c_i the running sum of the cell
 * counts of the cases before it; a case of dimension d uses rows 0 .. d+1,
 * (rho, rho u_1 .. rho u_d, E), and leaves the rows after them zero. */
typedef struct dvm_batch dvm_batch;

/* cfgs: ncases configurations (dim 1 or 2).  Device memory is allocated
 * with cudaMalloc and freed by dvm_batch_destroy.  DVM_ERR_ARG if a case is
 * invalid, a 2D case is not periodic or too large, or the cases disagree on
 * scheme or precision. */
int dvm_batch_create(const dvm_config* cfgs, int ncases, void* cuda_stream,
                     dvm_batch** out);
void dvm_batch_destroy(dvm_batch* b);
const char* dvm_batch_last_error(const dvm_batch* b);
/* Total cells and phase-space points of the batch. */
int dvm_batch_sizes(const dvm_batch* b, long long* cells, long long* points);
/* Rows R of the packed moments (3 or 4, see above). */
int dvm_batch_moment_rows(const dvm_batch* b, int* rows);
/* f^0 = E[U^0] for every case (Eq. minimMax); U packed as above, host or
 * device. */
int dvm_batch_set_state_moments(dvm_batch* b, const double* U, int on_device);
int dvm_batch_step(dvm_batch* b, int nsteps);
int dvm_batch_step_async(dvm_batch* b, int nsteps);
int dvm_batch_sync_status(dvm_batch* b);
/* Packed moments of all cases into the caller's buffer (host or device). */
int dvm_batch_moments(dvm_batch* b, double* out, int on_device);
/* Pipelined read-back of the packed moments (R x total cells FP64), with the
 * semantics of dvm_moments_async / dvm_moments_wait: snapshot on the device in
 * stream order, copy on a private stream, at most two in flight, the status
 * word as each ticket's snapshot found it. */
int dvm_batch_moments_async(dvm_batch* b, double* out, int on_device, long long* ticket);
int dvm_batch_moments_wait(dvm_batch* b, long long ticket);
/* f of case icase at its cell centres, N_v x N_cells FP64 (velocity-major,
 * velocities and cells x fastest), host buffer. */
int dvm_batch_get_f(dvm_batch* b, int icase, double* out);
/* Step index, per-case Euler sub-steps and alpha of the last step's first
 * sub-step (summed over the directions of a 2D case) (host arrays of ncases
 * entries; any pointer may be NULL). */
int dvm_batch_info(dvm_batch* b, long long* n, int* substeps, double* alpha);
/* Launch of the kinetic pass: threads per CTA (multiple of 32, <= 1024),
 * cells per thread (1..8), velocity chunks per case (1..4; a case takes at
 * most one chunk per 16 velocities; each chunk is its own work item writing
 * its own FP64 partial moment sums, added in chunk order at the end of the
 * step) and resident CTAs per SM (0 = as many as fit, else at most that many).
 * The chunking changes the order in which the partial sums are added, so
 * results can differ in the last bits of FP64 between launches. */
int dvm_batch_set_tiling(dvm_batch* b, int threads, int cells_per_thread, int vchunks,
                         int ctas_per_sm);
/* Times the kinetic pass of every candidate launch (threads 64/128/256 x 1
 * or 2 cells per thread x 1/2/4 velocity chunks x 0/2/4 CTAs per SM) on the
 * current state, restores f, keeps the fastest and returns it with its time
 * in ms.  Needs a state. */
int dvm_batch_autotune(dvm_batch* b, int* threads, int* cells_per_thread, int* vchunks,
                       int* ctas_per_sm, double* best_ms);
/* Runs nsteps steps launch by launch with CUDA events around the kinetic
 * pass; *ms receives its average time. */
int dvm_batch_kinetic_ms(dvm_batch* b, int nsteps, double* ms);

/* ------------------------------------------------------------------------
 * Learned regime path.
 *
 * Theorem 1 (Section 4.3.1) shows that as lambda -> 0 the HOFKS moments are
 * the MUSCL solution of the Euler system: near equilibrium the kinetic
 * update adds nothing.  A cell flagged as near equilibrium takes that form
 * for one step (HOFKS only, periodic or outflow, any precision):
 *   - its f^n is taken to be E[U^n] and its lambda to be 0: W = U^n feeds the
 *     Euler part there, and its pieces enter the transport as E_k[U^n] with
 *     weight 1 (no read of memory);
 *   - the kinetic pass does not write its pieces; after the step its f is
 *     E[U^{n+1}] by definition (dvm_get_f returns that);
 *   - a cell that was flagged and no longer is gets E[U] written into its
 *     pieces before its next kinetic update.
 * Moments stay exactly conservative.  The flags come from the caller
 * (DVM_LEARN_GIVEN) or from a 10-64-64-1 tanh network evaluated on ten local
 * features of U^n at the start of every step (DVM_LEARN_MLP):
 *   0 rho, 1 u_x, 2 u_y, 3 theta, 4 log10 tau,
 *   5 log10 K(tau sqrt(theta) |grad ln rho|), 6 log10 K(tau sqrt(theta) |grad ln theta|),
 *   7 log10 K(tau |div u|), 8 log10 K(tau |du_x/dy|), 9 log10 K(tau |du_y/dx|),
 * K(a) = max(a, 1e-12), central differences over the two neighbours along each
 * direction (boundary rule of the direction); u_y and y-derivatives are 0 in
 * 1D.  The network predicts log10(||f - E[U]||_1 / ||E[U]||_1) (discrete L1
 * over velocities); a cell is flagged when the prediction is below thr.
 * Every check_every steps a seeded sample of cells is checked: for each
 * sampled flagged cell the full kinetic update of the step is evaluated from
 * its (partly equilibrium) neighbours and the true one-step non-equilibrium
 * of the result is measured; if it is not below thr the cell and every cell
 * within veto_radius (Chebyshev distance) stay unflagged for the rest of the
 * run.  Flags on cells with lambda = 1 (tau = inf) are ignored.
 * ------------------------------------------------------------------------ */
#define DVM_NFEAT 10
#define DVM_MLP_HIDDEN 64
/* packed FP32 parameters, row-major: W1[64][10], b1[64], W2[64][64], b2[64],
 * W3[64], b3 */
#define DVM_MLP_NPARAM (64 * 10 + 64 + 64 * 64 + 64 + 64 + 1)

typedef enum { DVM_LEARN_OFF = 0, DVM_LEARN_GIVEN = 1, DVM_LEARN_MLP = 2 } dvm_learn_mode;

typedef struct {
  int mode;                /* dvm_learn_mode */
  int mlp_precision;       /* DVM_F32: FP32 on CUDA cores; DVM_BF16S: BF16
                              operands, FP32 accumulate, on the tensor cores */
  float thr;               /* flag when the predicted log10 non-equilibrium < thr */
  int check_every;         /* steps between checks; 0 = no checks */
  int check_samples;       /* cells drawn per check (1..65536) */
  int veto_radius;         /* Chebyshev radius unflagged around a failed check */
  unsigned long long seed; /* draws of the checked cells */
  float feat_shift[DVM_NFEAT];  /* network input x' = (x - shift) * scale */
  float feat_scale[DVM_NFEAT];
} dvm_learn_config;

typedef struct {
  long long steps;         /* learned steps taken */
  long long flagged;       /* cells flagged in the last step */
  long long flagged_total; /* sum over steps */
  long long materialised;  /* cells written back as E when unflagged */
  long long checks;        /* checks run */
  long long checked;       /* flagged cells checked */
  long long failed;        /* checked cells whose true value was not below thr */
  long long vetoed;        /* cells under a veto */
  double sum_abs_err;      /* sum over checked cells of |prediction - true| (MLP mode) */
  double max_abs_err;
  double max_true;         /* largest true value seen by a check */
} dvm_learn_stats;

/* Switches the learned path on (or off with mode DVM_LEARN_OFF) for the
 * following steps; allocates its buffers.  DVM_ERR_ARG for FKS, a bad mode or
 * precision; in MLP mode the network parameters must be set before a step. */
int dvm_learn_enable(dvm_handle* h, const dvm_learn_config* cfg);
/* Network parameters, host FP32 DVM_MLP_NPARAM values (copied). */
int dvm_learn_set_params(dvm_handle* h, const float* P);
/* GIVEN mode: host, N_c bytes (nonzero = flag), used by every following step
 * until replaced. */
int dvm_learn_set_flags(dvm_handle* h, const unsigned char* flags);
/* Flags used by the last step (host, N_c bytes). */
int dvm_learn_flags(dvm_handle* h, unsigned char* out);
/* Network predictions of the last step (host, N_c FP32; MLP mode). */
int dvm_learn_predictions(dvm_handle* h, float* out);
int dvm_learn_get_stats(dvm_handle* h, dvm_learn_stats* out);
/* One learned step that also checks the n given cells (host int64 indices)
 * as the periodic check does and writes their true one-step log10
 * non-equilibrium to out (host FP32; flagged or not); the veto rule applies
 * to those that were flagged. */
int dvm_learn_step_checked(dvm_handle* h, int n, const long long* cells, float* out);

/* The ten features of the current state, host FP32, sample-major
 * (out[c * 10 + i]); tau from the handle's configuration. */
int dvm_features(dvm_handle* h, float* out);
/* Label of the current state: log10(max(||f - E[U]||_1 / ||E[U]||_1, 1e-12))
 * per cell, host FP32, from the true f (stored pieces plus deferred term, or
 * E for flagged cells). */
int dvm_noneq(dvm_handle* h, float* out);

/* ---- the network on its own: training and inference on device data ---- */
typedef struct dvm_mlp dvm_mlp;
typedef struct {
  int epochs;
  int batch;               /* samples per Adam step */
  float lr, beta1, beta2, eps;
  unsigned long long seed; /* per-epoch shuffles */
} dvm_train_config;

/* precision: DVM_F32 (CUDA cores) or DVM_BF16S (tensor cores, BF16 operands,
 * FP32 accumulate, FP32 master weights). */
int dvm_mlp_create(int precision, void* cuda_stream, dvm_mlp** out);
void dvm_mlp_destroy(dvm_mlp* m);
int dvm_mlp_set_params(dvm_mlp* m, const float* P);  /* host FP32, resets Adam */
int dvm_mlp_get_params(dvm_mlp* m, float* P);        /* host FP32 */
/* y = net(X): X device FP32 n x 10 (sample-major), y device FP32 n. */
int dvm_mlp_forward(dvm_mlp* m, long long n, const float* X, float* y);
/* Mean squared error over n samples and its gradient (device FP64,
 * DVM_MLP_NPARAM values, overwritten); *loss on the host. */
int dvm_mlp_loss_grad(dvm_mlp* m, long long n, const float* X, const float* t, double* grad,
                      double* loss);
/* Adam on the mean squared error over the n samples (device X, t), shuffled
 * every epoch; *loss = mean loss of the last epoch. */
int dvm_mlp_train(dvm_mlp* m, long long n, const float* X, const float* t,
                  const dvm_train_config* cfg, double* loss);

/* Allocation-free equilibrium.  The paper has no counterpart to this entry
 * point: it exists for callers that cannot allocate device memory (a program
 * that runs within a fixed device-memory budget set up in advance, or a host
 * thread that must not enter the CUDA allocator, e.g. while other threads
 * capture graphs).  It computes the same f = E[U] as the initial state built
 * by dvm_set_state_moments (see dvm_get_f at step 0), with no handle and no
 * workspace: its scratch (a status word, (C C^T)^{-1} and the per-cell
 * equilibrium parameters) is a static device array of
 * DVM_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until
 * the process exits.  It calls no cudaMalloc or cudaFree and no allocating
 * library routine.
 *   cfg:    grid and velocity set (tau, scheme, precision and boundaries are
 *           ignored; the output is FP64).
 *   U:      device pointer, (d+2) x N_c FP64 moments, caller-owned.
 *   f:      device pointer, N_v x N_c FP64 output (velocity-major, cell
 *           positions), caller-owned.
 *   stream: cudaStream_t or NULL; the call synchronises it before returning.
 * Size limit: DVM_NOALLOC_HEADER_BYTES + 8 N_c (P + 1) bytes must fit in the
 * scratch, P the padded count of per-cell parameter rows (12 in 1D, 16 in 2D
 * and 3D), i.e. at most 61677 cells in 2D or 3D and 80654 in 1D; larger
 * problems return
 * DVM_ERR_TOO_LARGE without launching anything.  Returns DVM_ERR_NONPHYSICAL
 * or DVM_ERR_NONFINITE for bad moments, DVM_ERR_CUDA if a CUDA call fails.
 * The first call on each device looks up the device address of the scratch
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one scratch array, which
 * keeps the last call's contents; calls that overlap on the GPU (different
 * streams or host threads at once) race on it and must be serialised by the
 * caller. */
int dvm_equilibrium_noalloc(const dvm_config* cfg, const double* U, double* f,
                            void* cuda_stream);

/* Self-test of the device-side failure detection (no handle, no GPU fault):
 * runs one of the library's bounded waits on an event that never comes and
 * returns the device status word it left in *status, which is
 * DVM_ERR_TIMEOUT when the wait gave up as designed; the context stays
 * usable.
 *   which: DVM_SELFTEST_GRID_BARRIER -- the grid barrier of the Euler
 *            launches, one of two blocks leaving without arriving (about one
 *            second at 2 GHz);
 *          DVM_SELFTEST_MBARRIER -- the mbarrier wait of the tensor-core
 *            kernels on a barrier nobody arrives at (about one second).
 *   stream: cudaStream_t or NULL; the call synchronises it.
 * Returns 0, DVM_ERR_ARG for another `which`, DVM_ERR_OOM or DVM_ERR_CUDA. */
enum { DVM_SELFTEST_GRID_BARRIER = 0, DVM_SELFTEST_MBARRIER = 1 };
int dvm_selftest_timeout(int which, void* cuda_stream, int* status);

#ifdef __cplusplus
}
#endif
#endif
