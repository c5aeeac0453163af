/*
 * dvm_oracle.h -- plain FP64 CPU reference of the discrete-velocity BGK
 * scheme of Dimarco & Loubere, "Towards an ultra efficient kinetic scheme,
 * Part II: the high order case" (FKS of Section 4.2, HOFKS of Section 4.3).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the FP64 reference the GPU library is
 * compared against.  It is slow on purpose: every step is written in the
 * order the paper gives it, with no blocking, fusion or reordering, so that
 * it can be read against the paper line by line.  It shares no source with
 * the CUDA library and must never be linked into it.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Layouts (all FP64, all row-major, all owned by the caller):
 *   cells      c = x + nx[0]*(y + nx[1]*z)                 (x fastest)
 *   velocities k = kx + nv[0]*(ky + nv[1]*kz), v_i = (kmin_i + k_i) * dv
 *   moments    U[i*Nc + c], i = 0..d+1: (rho, rho*u_1..rho*u_d, E)
 *   f          f[k*Nc + c]: value of f_k at the centre of cell c (the
 *              oracle stores f at cell positions and moves it every step)
 */
#ifndef DVM_ORACLE_H
#define DVM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_NONFINITE (-4)
#define ORC_ERR_NONPHYSICAL (-5)

#define ORC_FKS 0
#define ORC_HOFKS 1
#define ORC_HOFKS_UNLIMITED 2
#define ORC_HOFKS_WENO 3 /* HOFKS with the WENO5 Euler solver of Section 4.3.3 */
#define ORC_FKS_STRANG 4 /* FKS with Strang splitting (Section 4.2) */

#define ORC_PERIODIC 0
#define ORC_OUTFLOW 1

typedef struct {
  int d;          /* space dimension = velocity dimension, 1..3 (Section 2) */
  int nx[3];      /* cells per dimension, unused dimensions = 1 */
  double dx;      /* uniform cell size (Section 4) */
  int bc[3];      /* ORC_PERIODIC or ORC_OUTFLOW, per dimension */
  int nv[3];      /* velocities per dimension, unused dimensions = 1 */
  int kmin[3];    /* lowest velocity index per dimension (Section 3) */
  double dv;      /* velocity step */
  int p;          /* v_k dt/dx = k/p, i.e. dt = dx/(p dv) */
  int scheme;     /* ORC_FKS, ORC_HOFKS, ORC_HOFKS_UNLIMITED */
  int subcycles;  /* Euler sub-steps per kinetic step; 0 = CFL rule (Eq. Time2) */
} orc_config;

typedef struct orc_state orc_state;

/* Offset of the piece of velocity component k after n steps:
 * round-half-up of k*n/p (pieces are half-open on the left). */
long long orc_offset(long long k, long long n, long long p);

/* C (rows m_k dv^d, (d+2) x Nv) and A = (C C^T)^{-1} ((d+2) x (d+2)). */
int orc_matrices(const orc_config* cfg, double* C, double* A);

/* Pointwise Maxwellian M_k[U] (Eq. M) for one cell's moments U[d+2]. */
int orc_maxwellian(const orc_config* cfg, const double* U, double* M);

/* Conservative discrete Maxwellian E_k[U] (Eq. minimMax). */
int orc_equilibrium(const orc_config* cfg, const double* U, double* E);

/* L2-closest vector to ftilde[Nv] with moments U (Eq. minim1). */
int orc_project(const orc_config* cfg, const double* ftilde, const double* U,
                double* f);

/* Euler flux F(U) along direction dir (Eq. sys1), gamma = 1 + 2/d. */
void orc_euler_flux(int d, const double* U, int dir, double* F);

/* Largest |u_dir| + sqrt(gamma*theta) over all cells, per direction. */
int orc_euler_alpha(const orc_config* cfg, const double* U, double* alpha);

/* One forward-Euler MUSCL sub-step (Eq. discmom), summed over directions:
 * Wout = W - dt/dx * sum_dir (psi_{+1/2} - psi_{-1/2}).  limited=0 sets the
 * limiter to 1. */
int orc_muscl_step(const orc_config* cfg, const double* W, double dt,
                   const double* alpha, int limited, double* Wout);

/* WENO5 interface values: out[j] = the left-biased value at j+1/2 of the
 * periodic samples v[0..n-1] (n >= 5); linear != 0 takes the optimal linear
 * weights instead of the nonlinear ones. */
int orc_weno5_reconstruct(const double* v, int n, int linear, double* out);

/* One Euler sub-step of length dt of the WENO5 scheme on the split fluxes
 * (F +- alpha U)/2 (alpha per direction), three-stage SSP Runge-Kutta. */
int orc_weno_step(const orc_config* cfg, const double* W, double dt,
                  const double* alpha, int linear, double* Wout);

/* Exact solution of the 1D Euler Riemann problem at the points xi = x/t. */
int orc_riemann_exact(double gamma, double rl, double ul, double pl,
                      double rr, double ur, double pr, const double* xi,
                      int npts, double* rho, double* u, double* pres,
                      double* pstar, double* ustar);

/* Scheme state. tau: per-cell relaxation times (Nc values) or NULL for the
 * uniform tau_uniform; INFINITY gives lambda = 1 exactly. */
orc_state* orc_create(const orc_config* cfg, const double* tau,
                      double tau_uniform);
void orc_destroy(orc_state* S);
/* f^0 = E[U^0] (Section 4.2, first step). */
int orc_set_moments(orc_state* S, const double* U);
int orc_step(orc_state* S, int nsteps);
void orc_get_moments(const orc_state* S, double* U);
void orc_get_f(const orc_state* S, double* f);
/* U_E, U_M and U_* of the last HOFKS step (Eqs. UK, mom). */
void orc_get_parts(const orc_state* S, double* UE, double* UM, double* Ustar);
/* dt, step index, Euler sub-steps and alpha of the last step. */
void orc_info(const orc_state* S, double* dt, long long* n, int* m,
              double* alpha);

/* ---- learned regime path (test reference of the flagged step) ---- */

/* One HOFKS step with the cells flags[c] != 0 treated as at equilibrium:
 * their f^n is E[U^n], their lambda 0 (the lambda -> 0 form of Theorem 1);
 * afterwards their f^{n+1} is E[U^{n+1}] unless keep_raw != 0.  Flags on
 * cells with lambda = 1 are ignored. */
int orc_step_flagged(orc_state* S, const unsigned char* flags, int keep_raw);

/* Replace the per-cell lambda of a state (Nc values). */
void orc_set_lambda(orc_state* S, const double* lam);

/* Deep copy of a scheme state. */
orc_state* orc_clone(const orc_state* S);

/* log10(max(||f_c - E[U_c]||_1 / ||E[U_c]||_1, 1e-12)) per cell. */
int orc_noneq(const orc_config* cfg, const double* f, const double* U, double* out);

/* The ten regime features per cell, out[i*Nc + c] (see dvm_oracle.c). */
int orc_features(const orc_config* cfg, const double* U, const double* tau, double* out);

#ifdef __cplusplus
}
#endif
#endif
