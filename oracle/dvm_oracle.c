/*
 * dvm_oracle.c -- plain FP64 CPU reference of FKS / HOFKS.
 *
 * TEST INFRASTRUCTURE ONLY (see dvm_oracle.h).  Written from the paper:
 *   Section 3       discrete velocity model, moments (Eq. DM)
 *   Section 4.1     conservative projection (Eqs. minim1, minimMax)
 *   Section 4.2     FKS: exact transport, then relaxation (Eq. relaxdvm);
 *                   the Strang splitting the section mentions as the more
 *                   accurate alternative: half relaxation, transport, half
 *                   relaxation
 *   Section 4.3.1   HOFKS: relaxation, transport, U_M replaced by U_E
 *                   (Eqs. UK, mom, cons, minim_full)
 *   Section 4.3.2   MUSCL finite volume Euler solver (Eq. discmom)
 *   Section 4.3.3   Euler time-step rule (Eq. Time2); the WENO solver the
 *                   section names as an alternative (finite-difference WENO5
 *                   of Jiang and Shu, as in Shu's 1998 lecture notes)
 * Readings where the paper is silent are marked "reading:" below.
 *
 * f is stored at cell positions and physically moved every step, the most
 * literal form of the exact transport; nothing here uses the piece-index
 * representation of the GPU library.
 */
#include "dvm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXM 5 /* d + 2 for d = 3 */

/* ------------------------------------------------------------------------ */
/* grid helpers                                                             */
/* ------------------------------------------------------------------------ */

static long ncells(const orc_config* g) {
  return (long)g->nx[0] * g->nx[1] * g->nx[2];
}
static long nvel(const orc_config* g) {
  return (long)g->nv[0] * g->nv[1] * g->nv[2];
}

static int check_config(const orc_config* g) {
  if (g->d < 1 || g->d > 3) return ORC_ERR_ARG;
  for (int i = 0; i < 3; ++i) {
    if (g->nx[i] < 1 || g->nv[i] < 1) return ORC_ERR_ARG;
    if (i >= g->d && (g->nx[i] != 1 || g->nv[i] != 1)) return ORC_ERR_ARG;
    if (g->bc[i] != ORC_PERIODIC && g->bc[i] != ORC_OUTFLOW) return ORC_ERR_ARG;
  }
  if (!(g->dx > 0) || !(g->dv > 0) || g->p < 1) return ORC_ERR_ARG;
  if (g->scheme < ORC_FKS || g->scheme > ORC_FKS_STRANG) return ORC_ERR_ARG;
  if (g->subcycles < 0) return ORC_ERR_ARG;
  return ORC_OK;
}

/* Velocity vector of linear index k (Section 3: v_k = k dv, a = 0). */
static void velocity(const orc_config* g, long k, double v[3]) {
  long kx = k % g->nv[0];
  long ky = (k / g->nv[0]) % g->nv[1];
  long kz = k / ((long)g->nv[0] * g->nv[1]);
  v[0] = (double)(g->kmin[0] + kx) * g->dv;
  v[1] = (g->d > 1) ? (double)(g->kmin[1] + ky) * g->dv : 0.0;
  v[2] = (g->d > 2) ? (double)(g->kmin[2] + kz) * g->dv : 0.0;
}

static void velocity_index(const orc_config* g, long k, long kk[3]) {
  kk[0] = g->kmin[0] + k % g->nv[0];
  kk[1] = g->kmin[1] + (k / g->nv[0]) % g->nv[1];
  kk[2] = g->kmin[2] + k / ((long)g->nv[0] * g->nv[1]);
}

static void cell_coords(const orc_config* g, long c, long xyz[3]) {
  xyz[0] = c % g->nx[0];
  xyz[1] = (c / g->nx[0]) % g->nx[1];
  xyz[2] = c / ((long)g->nx[0] * g->nx[1]);
}

static long cell_index(const orc_config* g, const long xyz[3]) {
  return xyz[0] + (long)g->nx[0] * (xyz[1] + (long)g->nx[1] * xyz[2]);
}

/* Apply the boundary rule to a coordinate that may lie outside [0, n):
 * periodic wraps, outflow clamps to the boundary cell (reading: zero-gradient
 * extrapolation, the paper does not state its boundary treatment). */
static long boundary(long x, long n, int bc) {
  if (bc == ORC_PERIODIC) {
    long r = x % n;
    return r < 0 ? r + n : r;
  }
  if (x < 0) return 0;
  if (x >= n) return n - 1;
  return x;
}

static long neighbour(const orc_config* g, long c, int dir, long off) {
  long xyz[3];
  cell_coords(g, c, xyz);
  xyz[dir] = boundary(xyz[dir] + off, g->nx[dir], g->bc[dir]);
  return cell_index(g, xyz);
}

/* ------------------------------------------------------------------------ */
/* exact transport offsets (Section 4.2)                                     */
/* ------------------------------------------------------------------------ */

/* The piece that started in cell j has moved by v_k t^n / dx = k n / p cells.
 * With pieces half-open on the left, (x_{j-1/2}, x_{j+1/2}], the cell centre
 * x_c lies in the piece j = c - floor(k n / p + 1/2).  Reading: the paper
 * does not say which piece owns a centre that falls on a piece boundary. */
long long orc_offset(long long k, long long n, long long p) {
  long long num = 2 * k * n + p;
  long long den = 2 * p;
  long long q = num / den;
  if ((num % den != 0) && ((num < 0) != (den < 0))) q -= 1;
  return q;
}

/* ------------------------------------------------------------------------ */
/* moments, C and (C C^T)^{-1} (Sections 3 and 4.1)                         */
/* ------------------------------------------------------------------------ */

/* Collision invariants m_k = (1, v_k, |v_k|^2 / 2) (Section 3). */
static void invariants(int d, const double v[3], double m[MAXM]) {
  m[0] = 1.0;
  double v2 = 0.0;
  for (int i = 0; i < d; ++i) {
    m[1 + i] = v[i];
    v2 += v[i] * v[i];
  }
  m[d + 1] = 0.5 * v2;
}

/* Inverse of a small symmetric positive definite matrix via Cholesky. */
static int spd_inverse(int n, const double* S, double* Sinv) {
  double L[MAXM * MAXM];
  memset(L, 0, sizeof L);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = S[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      if (i == j) {
        if (!(s > 0)) return ORC_ERR_ARG;
        L[i * n + i] = sqrt(s);
      } else {
        L[i * n + j] = s / L[j * n + j];
      }
    }
  }
  /* solve L L^T x = e_col for every unit vector */
  for (int col = 0; col < n; ++col) {
    double y[MAXM], x[MAXM];
    for (int i = 0; i < n; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
      x[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i) Sinv[i * n + col] = x[i];
  }
  return ORC_OK;
}

/* C has rows m_k dv^d (Section 4.1), A = (C C^T)^{-1}. */
int orc_matrices(const orc_config* g, double* C, double* A) {
  int rc = check_config(g);
  if (rc) return rc;
  const int d = g->d, nm = d + 2;
  const long nv = nvel(g);
  const double w = pow(g->dv, d);
  for (long k = 0; k < nv; ++k) {
    double v[3], m[MAXM];
    velocity(g, k, v);
    invariants(d, v, m);
    for (int i = 0; i < nm; ++i) C[i * nv + k] = m[i] * w;
  }
  double CCt[MAXM * MAXM];
  for (int i = 0; i < nm; ++i)
    for (int j = 0; j < nm; ++j) {
      double s = 0.0;
      for (long k = 0; k < nv; ++k) s += C[i * nv + k] * C[j * nv + k];
      CCt[i * nm + j] = s;
    }
  return spd_inverse(nm, CCt, A);
}

/* rho, u, theta from U (Eqs. Mo, E): E = rho|u|^2/2 + d rho theta / 2. */
static int primitives(int d, const double* U, double* rho, double u[3],
                      double* theta) {
  *rho = U[0];
  double u2 = 0.0;
  u[0] = u[1] = u[2] = 0.0;
  for (int i = 0; i < d; ++i) {
    u[i] = U[1 + i] / U[0];
    u2 += u[i] * u[i];
  }
  *theta = (2.0 * U[d + 1] / U[0] - u2) / d;
  for (int i = 0; i < d + 2; ++i)
    if (!isfinite(U[i])) return ORC_ERR_NONFINITE;
  if (!(*rho > 0) || !(*theta > 0)) return ORC_ERR_NONPHYSICAL;
  return ORC_OK;
}

/* Pointwise Maxwellian (Eq. M) at every discrete velocity, R = 1. */
int orc_maxwellian(const orc_config* g, const double* U, double* M) {
  const int d = g->d;
  double rho, u[3], theta;
  int rc = primitives(d, U, &rho, u, &theta);
  if (rc) return rc;
  const double pref = rho / pow(2.0 * M_PI * theta, 0.5 * d);
  const long nv = nvel(g);
  for (long k = 0; k < nv; ++k) {
    double v[3], q = 0.0;
    velocity(g, k, v);
    for (int i = 0; i < d; ++i) q += (v[i] - u[i]) * (v[i] - u[i]);
    M[k] = pref * exp(-q / (2.0 * theta));
  }
  return ORC_OK;
}

/* f = ftilde + C^T A (U - C ftilde)   (Eq. minim1). */
static void project_with(int nm, long nv, const double* C, const double* A,
                         const double* ftilde, const double* U, double* f) {
  double r[MAXM], mu[MAXM];
  for (int i = 0; i < nm; ++i) {
    double s = 0.0;
    for (long k = 0; k < nv; ++k) s += C[i * nv + k] * ftilde[k];
    r[i] = U[i] - s;
  }
  for (int i = 0; i < nm; ++i) {
    double s = 0.0;
    for (int j = 0; j < nm; ++j) s += A[i * nm + j] * r[j];
    mu[i] = s;
  }
  for (long k = 0; k < nv; ++k) {
    double s = 0.0;
    for (int i = 0; i < nm; ++i) s += C[i * nv + k] * mu[i];
    f[k] = ftilde[k] + s;
  }
}

int orc_project(const orc_config* g, const double* ftilde, const double* U,
                double* f) {
  int rc = check_config(g);
  if (rc) return rc;
  const int nm = g->d + 2;
  const long nv = nvel(g);
  double* C = malloc(sizeof(double) * nm * nv);
  double A[MAXM * MAXM];
  if (!C) return ORC_ERR_OOM;
  rc = orc_matrices(g, C, A);
  if (!rc) project_with(nm, nv, C, A, ftilde, U, f);
  free(C);
  return rc;
}

/* E[U] = M[U] + C^T A (U - C M[U])   (Eq. minimMax). */
static int equilibrium_with(const orc_config* g, const double* C,
                            const double* A, const double* U, double* M,
                            double* E) {
  int rc = orc_maxwellian(g, U, M);
  if (rc) return rc;
  project_with(g->d + 2, nvel(g), C, A, M, U, E);
  return ORC_OK;
}

int orc_equilibrium(const orc_config* g, const double* U, double* E) {
  int rc = check_config(g);
  if (rc) return rc;
  const int nm = g->d + 2;
  const long nv = nvel(g);
  double* C = malloc(sizeof(double) * nm * nv);
  double* M = malloc(sizeof(double) * nv);
  double A[MAXM * MAXM];
  if (!C || !M) {
    free(C);
    free(M);
    return ORC_ERR_OOM;
  }
  rc = orc_matrices(g, C, A);
  if (!rc) rc = equilibrium_with(g, C, A, U, M, E);
  free(C);
  free(M);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Euler system and MUSCL (Sections 2, 4.3.2, 4.3.3)                         */
/* ------------------------------------------------------------------------ */

/* Flux of Eq. sys1 along dir.  p = rho theta and E = d/2 rho theta +
 * rho|u|^2/2 give p = (2/d)(E - rho|u|^2/2), i.e. gamma = 1 + 2/d.
 * A cell with zero density carries no flux (reading: only reached when
 * lambda = 1 makes W = 0). */
void orc_euler_flux(int d, const double* U, int dir, double* F) {
  const double rho = U[0];
  double u[3] = {0.0, 0.0, 0.0}, ke = 0.0;
  if (rho != 0.0) {
    for (int j = 0; j < d; ++j) {
      u[j] = U[1 + j] / rho;
      ke += 0.5 * U[1 + j] * u[j];
    }
  }
  const double p = (2.0 / d) * (U[d + 1] - ke);
  F[0] = U[1 + dir];
  for (int j = 0; j < d; ++j) F[1 + j] = U[1 + j] * u[dir] + (j == dir ? p : 0.0);
  F[d + 1] = (U[d + 1] + p) * u[dir];
}

/* alpha_dir = max over cells of |u_dir| + c, c = sqrt(gamma theta): the
 * largest eigenvalue of the Euler system along dir (reading: one global alpha
 * per direction per kinetic step). */
int orc_euler_alpha(const orc_config* g, const double* U, double* alpha) {
  const int d = g->d, nm = d + 2;
  const long nc = ncells(g);
  const double gamma = 1.0 + 2.0 / d;
  for (int i = 0; i < 3; ++i) alpha[i] = 0.0;
  for (long c = 0; c < nc; ++c) {
    double Uc[MAXM], rho, u[3], theta;
    for (int i = 0; i < nm; ++i) Uc[i] = U[i * nc + c];
    int rc = primitives(d, Uc, &rho, u, &theta);
    if (rc) return rc;
    const double cs = sqrt(gamma * theta);
    for (int i = 0; i < d; ++i) {
      double a = fabs(u[i]) + cs;
      if (a > alpha[i]) alpha[i] = a;
    }
  }
  return ORC_OK;
}

/* van Leer slope of Section 4.3.2: b * phi(a/b), phi(chi) = (|chi|+chi)/(1+chi),
 * written in product form so that b = 0 and a = -b give zero (reading). */
static double limited_slope(double a, double b, int limited) {
  if (!limited) return b;
  if (a * b > 0.0) return (fabs(a) * fabs(b) + a * b) / (a + b);
  return 0.0;
}

/* psi_{j+1/2} of Eq. discmom along dir, from cells jm1, j, jp1, jp2. */
static void muscl_face_flux(const orc_config* g, const double* W, long jm1,
                            long j, long jp1, long jp2, int dir, double alpha,
                            int limited, double* psi) {
  const int d = g->d, nm = d + 2;
  const long nc = ncells(g);
  double Us[4][MAXM], Fs[4][MAXM];
  long idx[4] = {jm1, j, jp1, jp2};
  for (int s = 0; s < 4; ++s) {
    for (int i = 0; i < nm; ++i) Us[s][i] = W[i * nc + idx[s]];
    orc_euler_flux(d, Us[s], dir, Fs[s]);
  }
  for (int i = 0; i < nm; ++i) {
    double Gp[4], Gm[4];
    for (int s = 0; s < 4; ++s) {
      Gp[s] = Fs[s][i] + alpha * Us[s][i];
      Gm[s] = Fs[s][i] - alpha * Us[s][i];
    }
    /* sigma^+_j: chi^+_j = (G+_j - G+_{j-1}) / (G+_{j+1} - G+_j) */
    const double sp = limited_slope(Gp[1] - Gp[0], Gp[2] - Gp[1], limited);
    /* sigma^-_{j+1}: chi^-_{j+1} = (G-_{j+1} - G-_j) / (G-_{j+2} - G-_{j+1}) */
    const double sm = limited_slope(Gm[2] - Gm[1], Gm[3] - Gm[2], limited);
    psi[i] = 0.5 * (Fs[1][i] + Fs[2][i]) - 0.5 * alpha * (Us[2][i] - Us[1][i]) +
             0.25 * (sp - sm);
  }
}

/* One forward-Euler step of Eq. discmom; in several dimensions the flux
 * differences of all directions are summed (reading: unsplit). */
int orc_muscl_step(const orc_config* g, const double* W, double dt,
                   const double* alpha, int limited, double* Wout) {
  const int d = g->d, nm = d + 2;
  const long nc = ncells(g);
  for (long c = 0; c < nc; ++c) {
    double acc[MAXM] = {0};
    for (int dir = 0; dir < d; ++dir) {
      const long m2 = neighbour(g, c, dir, -2), m1 = neighbour(g, c, dir, -1);
      const long p1 = neighbour(g, c, dir, 1), p2 = neighbour(g, c, dir, 2);
      double psi_r[MAXM], psi_l[MAXM];
      muscl_face_flux(g, W, m1, c, p1, p2, dir, alpha[dir], limited, psi_r);
      muscl_face_flux(g, W, m2, m1, c, p1, dir, alpha[dir], limited, psi_l);
      for (int i = 0; i < nm; ++i) acc[i] += psi_r[i] - psi_l[i];
    }
    for (int i = 0; i < nm; ++i) Wout[i * nc + c] = W[i * nc + c] - dt / g->dx * acc[i];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* WENO Euler solver (Section 4.3.3 names WENO as a higher-order alternative  */
/* to MUSCL; reading: the finite-difference WENO5 scheme of Jiang and Shu,    */
/* component by component, on the Lax-Friedrichs split fluxes                 */
/* f+- = (F +- alpha U) / 2 with the same global alpha per direction as the   */
/* MUSCL flux, advanced by the three-stage SSP Runge-Kutta scheme of Shu and  */
/* Osher over each Euler sub-step of Eq. Time2 length)                        */
/* ------------------------------------------------------------------------ */

/* Interface value at j+1/2 from v[0..4] = values at j-2 .. j+2, biased to the
 * left (upwind for a right-moving flux).  Three candidate quadratics on the
 * sub-stencils {j-2, j-1, j}, {j-1, j, j+1}, {j, j+1, j+2}, each third-order
 * accurate at j+1/2, blended with weights d_k / (eps + beta_k)^2 normalised
 * to one, beta_k the smoothness indicators (sums of squared scaled
 * derivatives of the candidate over the cell); linear != 0 uses the optimal
 * weights d = (1/10, 6/10, 3/10) themselves (fifth order, no limiting). */
static double weno5_left(const double* v, int linear) {
  const double q0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
  const double q1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
  const double q2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
  const double d0 = 0.1, d1 = 0.6, d2 = 0.3;
  if (linear) return d0 * q0 + d1 * q1 + d2 * q2;
  const double a0 = v[0] - 2.0 * v[1] + v[2], b0 = v[0] - 4.0 * v[1] + 3.0 * v[2];
  const double a1 = v[1] - 2.0 * v[2] + v[3], b1 = v[1] - v[3];
  const double a2 = v[2] - 2.0 * v[3] + v[4], b2 = 3.0 * v[2] - 4.0 * v[3] + v[4];
  const double beta0 = 13.0 / 12.0 * a0 * a0 + 0.25 * b0 * b0;
  const double beta1 = 13.0 / 12.0 * a1 * a1 + 0.25 * b1 * b1;
  const double beta2 = 13.0 / 12.0 * a2 * a2 + 0.25 * b2 * b2;
  const double eps = 1e-6;
  const double w0 = d0 / ((eps + beta0) * (eps + beta0));
  const double w1 = d1 / ((eps + beta1) * (eps + beta1));
  const double w2 = d2 / ((eps + beta2) * (eps + beta2));
  return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}

int orc_weno5_reconstruct(const double* v, int n, int linear, double* out) {
  if (!v || !out || n < 5) return ORC_ERR_ARG;
  for (int j = 0; j < n; ++j) {
    double s[5];
    for (int o = 0; o < 5; ++o) s[o] = v[(j + o - 2 + n) % n];
    out[j] = weno5_left(s, linear);
  }
  return ORC_OK;
}

/* psi_{j+1/2} along dir from the cells jm2 .. jp3 (indices in c[0..5]): the
 * left-biased value of f+ from j-2 .. j+2 plus the right-biased value of f-
 * from j+3 .. j-1 (the same formula on the mirrored stencil). */
static void weno_face_flux(const orc_config* g, const double* W, const long* c, int dir,
                           double alpha, int linear, double* psi) {
  const int d = g->d, nm = d + 2;
  const long nc = ncells(g);
  double Us[6][MAXM], Fs[6][MAXM];
  for (int s = 0; s < 6; ++s) {
    for (int i = 0; i < nm; ++i) Us[s][i] = W[i * nc + c[s]];
    orc_euler_flux(d, Us[s], dir, Fs[s]);
  }
  for (int i = 0; i < nm; ++i) {
    double fp[5], fm[5];
    for (int s = 0; s < 5; ++s) {
      fp[s] = 0.5 * (Fs[s][i] + alpha * Us[s][i]);          /* cells j-2 .. j+2 */
      fm[s] = 0.5 * (Fs[5 - s][i] - alpha * Us[5 - s][i]);  /* cells j+3 .. j-1 */
    }
    psi[i] = weno5_left(fp, linear) + weno5_left(fm, linear);
  }
}

/* L(W) = -(1/dx) sum_dir (psi_{j+1/2} - psi_{j-1/2}) (reading: unsplit). */
static void weno_rhs(const orc_config* g, const double* W, const double* alpha, int linear,
                     double* L) {
  const int d = g->d, nm = d + 2;
  const long nc = ncells(g);
  for (long c = 0; c < nc; ++c) {
    double acc[MAXM] = {0};
    for (int dir = 0; dir < d; ++dir) {
      long st[7];
      for (int o = 0; o < 7; ++o) st[o] = neighbour(g, c, dir, o - 3);  /* j-3 .. j+3 */
      double pr[MAXM], pl[MAXM];
      weno_face_flux(g, W, st + 1, dir, alpha[dir], linear, pr);  /* j+1/2: j-2 .. j+3 */
      weno_face_flux(g, W, st, dir, alpha[dir], linear, pl);      /* j-1/2: j-3 .. j+2 */
      for (int i = 0; i < nm; ++i) acc[i] += pr[i] - pl[i];
    }
    for (int i = 0; i < nm; ++i) L[i * nc + c] = -acc[i] / g->dx;
  }
}

/* One Euler sub-step of length dt by the three-stage SSP Runge-Kutta scheme:
 *   W1 = W + dt L(W)
 *   W2 = 3/4 W + 1/4 (W1 + dt L(W1))
 *   W' = 1/3 W + 2/3 (W2 + dt L(W2))
 * with alpha (per direction) held for the three stages. */
int orc_weno_step(const orc_config* g, const double* W, double dt, const double* alpha,
                  int linear, double* Wout) {
  const int nm = g->d + 2;
  const long nc = ncells(g), n = nm * nc;
  double* L = malloc(sizeof(double) * n);
  double* W1 = calloc(n, sizeof(double));
  double* W2 = calloc(n, sizeof(double));
  if (!L || !W1 || !W2) {
    free(L);
    free(W1);
    free(W2);
    return ORC_ERR_OOM;
  }
  weno_rhs(g, W, alpha, linear, L);
  for (long i = 0; i < n; ++i) W1[i] = W[i] + dt * L[i];
  weno_rhs(g, W1, alpha, linear, L);
  for (long i = 0; i < n; ++i) W2[i] = 0.75 * W[i] + 0.25 * (W1[i] + dt * L[i]);
  weno_rhs(g, W2, alpha, linear, L);
  for (long i = 0; i < n; ++i) Wout[i] = W[i] / 3.0 + 2.0 / 3.0 * (W2[i] + dt * L[i]);
  free(L);
  free(W1);
  free(W2);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* scheme state                                                             */
/* ------------------------------------------------------------------------ */

struct orc_state {
  orc_config g;
  int nm;
  long nc, nv;
  double dt;
  double* C;     /* nm x nv */
  double A[MAXM * MAXM];
  double* lam;   /* nc: lambda = exp(-dt/tau) */
  double* lamh;  /* nc: exp(-dt/(2 tau)), the half step of the Strang splitting */
  double* f;     /* nv x nc at cell positions */
  double* fnew;  /* nv x nc */
  double* U;     /* nm x nc */
  double* Eq;    /* nv x nc: E_k[U_s] of the step */
  double* UE;    /* nm x nc */
  double* UM;    /* nm x nc */
  double* Us;    /* nm x nc */
  double* W0;    /* nm x nc, MUSCL buffers */
  double* W1;
  double* tmpM;  /* nv */
  double* tmpF;  /* nv */
  long long n;
  int last_m;
  double alpha[3];
};

void orc_destroy(orc_state* S) {
  if (!S) return;
  free(S->C);
  free(S->lam);
  free(S->lamh);
  free(S->f);
  free(S->fnew);
  free(S->U);
  free(S->Eq);
  free(S->UE);
  free(S->UM);
  free(S->Us);
  free(S->W0);
  free(S->W1);
  free(S->tmpM);
  free(S->tmpF);
  free(S);
}

orc_state* orc_create(const orc_config* g, const double* tau,
                      double tau_uniform) {
  if (check_config(g)) return NULL;
  orc_state* S = calloc(1, sizeof(orc_state));
  if (!S) return NULL;
  S->g = *g;
  S->nm = g->d + 2;
  S->nc = ncells(g);
  S->nv = nvel(g);
  /* v_k dt / dx = k / p  (integer shifts for p = 1) */
  S->dt = g->dx / (g->p * g->dv);
  const size_t phase = sizeof(double) * (size_t)S->nc * (size_t)S->nv;
  const size_t mom = sizeof(double) * (size_t)S->nc * (size_t)S->nm;
  S->C = malloc(sizeof(double) * S->nm * S->nv);
  S->lam = malloc(sizeof(double) * S->nc);
  S->lamh = malloc(sizeof(double) * S->nc);
  S->f = calloc(1, phase);
  S->fnew = calloc(1, phase);
  S->Eq = calloc(1, phase);
  S->U = calloc(1, mom);
  S->UE = calloc(1, mom);
  S->UM = calloc(1, mom);
  S->Us = calloc(1, mom);
  S->W0 = calloc(1, mom);
  S->W1 = calloc(1, mom);
  S->tmpM = malloc(sizeof(double) * S->nv);
  S->tmpF = malloc(sizeof(double) * S->nv);
  if (!S->C || !S->lam || !S->lamh || !S->f || !S->fnew || !S->Eq || !S->U || !S->UE ||
      !S->UM || !S->Us || !S->W0 || !S->W1 || !S->tmpM || !S->tmpF ||
      orc_matrices(g, S->C, S->A)) {
    orc_destroy(S);
    return NULL;
  }
  /* lambda = exp(-dt/tau) (Section 4.3.1); tau = inf gives exactly 1. */
  for (long c = 0; c < S->nc; ++c) {
    const double t = tau ? tau[c] : tau_uniform;
    S->lam[c] = exp(-S->dt / t);
    S->lamh[c] = exp(-S->dt / (2.0 * t));
  }
  return S;
}

int orc_set_moments(orc_state* S, const double* U) {
  memcpy(S->U, U, sizeof(double) * S->nm * S->nc);
  double Uc[MAXM];
  for (long c = 0; c < S->nc; ++c) {
    for (int i = 0; i < S->nm; ++i) Uc[i] = U[i * S->nc + c];
    int rc = equilibrium_with(&S->g, S->C, S->A, Uc, S->tmpM, S->tmpF);
    if (rc) return rc;
    for (long k = 0; k < S->nv; ++k) S->f[k * S->nc + c] = S->tmpF[k];
  }
  S->n = 0;
  return ORC_OK;
}

void orc_get_moments(const orc_state* S, double* U) {
  memcpy(U, S->U, sizeof(double) * S->nm * S->nc);
}
void orc_get_f(const orc_state* S, double* f) {
  memcpy(f, S->f, sizeof(double) * S->nv * S->nc);
}
void orc_get_parts(const orc_state* S, double* UE, double* UM, double* Ustar) {
  const size_t b = sizeof(double) * S->nm * S->nc;
  if (UE) memcpy(UE, S->UE, b);
  if (UM) memcpy(UM, S->UM, b);
  if (Ustar) memcpy(Ustar, S->Us, b);
}
void orc_info(const orc_state* S, double* dt, long long* n, int* m,
              double* alpha) {
  if (dt) *dt = S->dt;
  if (n) *n = S->n;
  if (m) *m = S->last_m;
  if (alpha)
    for (int i = 0; i < 3; ++i) alpha[i] = S->alpha[i];
}

/* Cell where the value seen at the centre of cell c after the step, for
 * velocity k, sat at time t^n: c - delta_k with delta the change of the
 * offsets over the step; boundary rule applied per dimension. */
static long source_cell(const orc_state* S, long c, long k) {
  const orc_config* g = &S->g;
  long xyz[3], kk[3];
  cell_coords(g, c, xyz);
  velocity_index(g, k, kk);
  for (int i = 0; i < g->d; ++i) {
    const long long delta =
        orc_offset(kk[i], S->n + 1, g->p) - orc_offset(kk[i], S->n, g->p);
    xyz[i] = boundary(xyz[i] - (long)delta, g->nx[i], g->bc[i]);
  }
  return cell_index(g, xyz);
}

/* E_k[U_s] for every cell s (Eq. minimMax), into S->Eq. */
static int equilibria(orc_state* S, const double* U) {
  double Uc[MAXM];
  for (long c = 0; c < S->nc; ++c) {
    for (int i = 0; i < S->nm; ++i) Uc[i] = U[i * S->nc + c];
    int rc = equilibrium_with(&S->g, S->C, S->A, Uc, S->tmpM, S->tmpF);
    if (rc) return rc;
    for (long k = 0; k < S->nv; ++k) S->Eq[k * S->nc + c] = S->tmpF[k];
  }
  return ORC_OK;
}

/* alpha of an Euler state W (flux splitting and Eq. Time2): per direction the
 * largest |u_dir| + sqrt(gamma theta) over the cells; cells with zero density
 * (lambda = 1 makes W = 0 there) carry no wave and are skipped. */
static void state_alpha(const orc_config* g, const double* W, double alpha[3]) {
  const int d = g->d, nm = d + 2;
  const long nc = ncells(g);
  const double gamma = 1.0 + 2.0 / d;
  for (int i = 0; i < 3; ++i) alpha[i] = 0.0;
  for (long c = 0; c < nc; ++c) {
    double Uc[MAXM] = {0.0, 0.0, 0.0, 0.0, 0.0}, rho, u[3], theta;
    for (int i = 0; i < nm; ++i) Uc[i] = W[i * nc + c];
    if (Uc[0] == 0.0) continue;
    primitives(d, Uc, &rho, u, &theta);
    const double cs = sqrt(gamma * theta);
    for (int i = 0; i < d; ++i) {
      const double a = fabs(u[i]) + cs;
      if (a > alpha[i]) alpha[i] = a;
    }
  }
}

/* U_E from W = (1 - lambda) U^n by MUSCL sub-steps covering the kinetic step
 * (Section 4.3.2).  Reading: U_E carries the (1 - lambda) weight so that
 * U_H = U_* + U_E has the mass of f; for uniform lambda this equals
 * (1 - lambda) MUSCL(U^n).  Each Euler sub-step takes alpha from its own
 * initial state and its length from Eq. Time2, dt_E = dx / (2 sum_i alpha_i)
 * (reading: unsplit multi-D), the last one shortened to end at dt; with a
 * fixed count m the sub-steps are dt/m long and alpha is still taken per
 * sub-step. */
static int euler_part(orc_state* S) {
  const long nc = S->nc;
  const int nm = S->nm;
  int all_free = 1;
  for (long c = 0; c < nc; ++c)
    if (S->lam[c] != 1.0) all_free = 0;
  if (all_free) {
    /* free transport: W = 0 and the Euler solve is skipped */
    memset(S->UE, 0, sizeof(double) * nm * nc);
    for (int i = 0; i < 3; ++i) S->alpha[i] = 0.0;
    S->last_m = 0;
    return ORC_OK;
  }
  for (int i = 0; i < nm; ++i)
    for (long c = 0; c < nc; ++c)
      S->W0[i * nc + c] = (1.0 - S->lam[c]) * S->U[i * nc + c];
  const int limited = (S->g.scheme == ORC_HOFKS);
  double* a = S->W0;
  double* b = S->W1;
  double t = 0.0;
  int m = 0;
  for (;;) {
    double alpha[3], asum = 0.0;
    state_alpha(&S->g, a, alpha);
    for (int i = 0; i < S->g.d; ++i) asum += alpha[i];
    if (m == 0)
      for (int i = 0; i < 3; ++i) S->alpha[i] = alpha[i];
    double dtE;
    int last;
    if (S->g.subcycles > 0) {
      dtE = S->dt / S->g.subcycles;
      last = (m + 1 == S->g.subcycles);
    } else {
      if (!(asum > 0.0)) return ORC_ERR_NONPHYSICAL;
      const double cfl = 0.5 * S->g.dx / asum;
      const double rem = S->dt - t;
      last = (cfl >= rem);
      dtE = last ? rem : cfl;
    }
    if (S->g.scheme == ORC_HOFKS_WENO) {
      const int rc = orc_weno_step(&S->g, a, dtE, alpha, 0, b);
      if (rc) return rc;
    } else {
      orc_muscl_step(&S->g, a, dtE, alpha, limited, b);
    }
    double* tmp = a;
    a = b;
    b = tmp;
    t += dtE;
    m += 1;
    if (last) break;
    if (m > 1000000) return ORC_ERR_NONPHYSICAL;
  }
  S->last_m = m;
  memcpy(S->UE, a, sizeof(double) * nm * nc);
  return ORC_OK;
}

/* HOFKS step (Section 4.3.1):
 *   f*      = lambda f^n + (1 - lambda) E^n            (relaxation first)
 *   U_K     = P(T(lambda f^n)) + P(T((1-lambda) E^n)) = U_* + U_M  (Eq. UK)
 *   U_H     = U_* + U_E                                 (Eq. mom)
 *   T'      = T((1-lambda)E^n) + C^T A (U_E - U_M)      (Eq. minim_full)
 *   f^{n+1} = T(lambda f^n) + T'                        */
static int step_hofks(orc_state* S) {
  const long nc = S->nc, nv = S->nv;
  const int nm = S->nm;
  int rc = euler_part(S);
  if (rc) return rc;
  rc = equilibria(S, S->U);
  if (rc) return rc;
  double* fstar = S->tmpF;
  for (long c = 0; c < nc; ++c) {
    double us[MAXM] = {0}, um[MAXM] = {0};
    for (long k = 0; k < nv; ++k) {
      const long s = source_cell(S, c, k);
      const double a = S->lam[s] * S->f[k * nc + s];
      const double b = (1.0 - S->lam[s]) * S->Eq[k * nc + s];
      for (int i = 0; i < nm; ++i) {
        us[i] += S->C[i * nv + k] * a;
        um[i] += S->C[i * nv + k] * b;
      }
      fstar[k] = a + b;
    }
    double r[MAXM], nu[MAXM];
    for (int i = 0; i < nm; ++i) r[i] = S->UE[i * nc + c] - um[i];
    for (int i = 0; i < nm; ++i) {
      double s = 0.0;
      for (int j = 0; j < nm; ++j) s += S->A[i * nm + j] * r[j];
      nu[i] = s;
    }
    for (long k = 0; k < nv; ++k) {
      double s = 0.0;
      for (int i = 0; i < nm; ++i) s += S->C[i * nv + k] * nu[i];
      S->fnew[k * nc + c] = fstar[k] + s;
    }
    for (int i = 0; i < nm; ++i) {
      S->Us[i * nc + c] = us[i];
      S->UM[i * nc + c] = um[i];
    }
  }
  for (int i = 0; i < nm; ++i)
    for (long c = 0; c < nc; ++c)
      S->U[i * nc + c] = S->Us[i * nc + c] + S->UE[i * nc + c];
  double* t = S->f;
  S->f = S->fnew;
  S->fnew = t;
  return ORC_OK;
}

/* FKS step (Section 4.2, generic time step): exact transport, moments of the
 * transported f at the cell centres, relaxation towards E[U*] (Eq. relaxdvm).
 * The relaxation acts at time t^{n+1}, at the cell the piece now occupies. */
static int step_fks(orc_state* S) {
  const long nc = S->nc, nv = S->nv;
  const int nm = S->nm;
  for (long c = 0; c < nc; ++c)
    for (long k = 0; k < nv; ++k)
      S->fnew[k * nc + c] = S->f[k * nc + source_cell(S, c, k)];
  for (long c = 0; c < nc; ++c)
    for (int i = 0; i < nm; ++i) {
      double s = 0.0;
      for (long k = 0; k < nv; ++k) s += S->C[i * nv + k] * S->fnew[k * nc + c];
      S->U[i * nc + c] = s;
    }
  int rc = equilibria(S, S->U);
  if (rc) return rc;
  for (long k = 0; k < nv; ++k)
    for (long c = 0; c < nc; ++c) {
      const double l = S->lam[c];
      S->fnew[k * nc + c] = l * S->fnew[k * nc + c] + (1.0 - l) * S->Eq[k * nc + c];
    }
  double* t = S->f;
  S->f = S->fnew;
  S->fnew = t;
  S->last_m = 0;
  return ORC_OK;
}

/* Relaxation over half a step at every cell (Eq. relaxdvm over dt/2):
 * f <- lambda_h f + (1 - lambda_h) E[U], U the moments of f at the cell,
 * lambda_h = exp(-dt/(2 tau)).  Leaves U in S->U. */
static int relax_half(orc_state* S) {
  const long nc = S->nc, nv = S->nv;
  const int nm = S->nm;
  for (long c = 0; c < nc; ++c)
    for (int i = 0; i < nm; ++i) {
      double s = 0.0;
      for (long k = 0; k < nv; ++k) s += S->C[i * nv + k] * S->f[k * nc + c];
      S->U[i * nc + c] = s;
    }
  int rc = equilibria(S, S->U);
  if (rc) return rc;
  for (long k = 0; k < nv; ++k)
    for (long c = 0; c < nc; ++c) {
      const double l = S->lamh[c];
      S->f[k * nc + c] = l * S->f[k * nc + c] + (1.0 - l) * S->Eq[k * nc + c];
    }
  return ORC_OK;
}

/* FKS with Strang splitting (Section 4.2 names it as the alternative to the
 * first-order splitting): relaxation over dt/2, exact transport over dt,
 * relaxation over dt/2. */
static int step_fks_strang(orc_state* S) {
  const long nc = S->nc, nv = S->nv;
  int rc = relax_half(S);
  if (rc) return rc;
  for (long c = 0; c < nc; ++c)
    for (long k = 0; k < nv; ++k)
      S->fnew[k * nc + c] = S->f[k * nc + source_cell(S, c, k)];
  double* t = S->f;
  S->f = S->fnew;
  S->fnew = t;
  rc = relax_half(S);
  S->last_m = 0;
  return rc;
}

int orc_step(orc_state* S, int nsteps) {
  for (int s = 0; s < nsteps; ++s) {
    int rc = (S->g.scheme == ORC_FKS)          ? step_fks(S)
             : (S->g.scheme == ORC_FKS_STRANG) ? step_fks_strang(S)
                                               : step_hofks(S);
    if (rc) return rc;
    S->n += 1;
    for (long c = 0; c < S->nc; ++c) {
      double Uc[MAXM], rho, u[3], theta;
      for (int i = 0; i < S->nm; ++i) Uc[i] = S->U[i * S->nc + c];
      rc = primitives(S->g.d, Uc, &rho, u, &theta);
      if (rc) return rc;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* learned regime path: flagged near-equilibrium cells                      */
/* ------------------------------------------------------------------------ */

/* One HOFKS step in which the cells with flags[c] != 0 are treated as being at
 * equilibrium.  Theorem 1 (Section 4.3.1) shows that the HOFKS moments reduce
 * to the MUSCL solution of the Euler system as lambda -> 0; a flagged cell
 * takes that form:
 *   (i)   its f^n is taken to be E[U^n_c] and its lambda to be 0;
 *   (ii)  the HOFKS step runs with this lambda field (W = (1 - lambda) U^n
 *         becomes U^n at flagged cells; their pieces enter the transport as
 *         E_k[U^n_c] with weight 1);
 *   (iii) afterwards the f^{n+1} of every flagged cell is E[U^{n+1}_c]
 *         (keep_raw = 0), or the raw f^{n+1} of the kinetic update is kept
 *         (keep_raw = 1: the one-step check of a flag).
 * A flag on a cell with lambda = 1 (tau = inf) is ignored.  HOFKS only. */
int orc_step_flagged(orc_state* S, const unsigned char* flags, int keep_raw) {
  if (S->g.scheme == ORC_FKS || S->g.scheme == ORC_FKS_STRANG) return ORC_ERR_ARG;
  const long nc = S->nc, nv = S->nv;
  const int nm = S->nm;
  double* lam_eff = malloc(sizeof(double) * nc);
  if (!lam_eff) return ORC_ERR_OOM;
  double Uc[MAXM];
  int rc = ORC_OK;
  for (long c = 0; c < nc; ++c) {
    const int fl = flags[c] != 0 && S->lam[c] != 1.0;
    lam_eff[c] = fl ? 0.0 : S->lam[c];
    if (!fl) continue;
    for (int i = 0; i < nm; ++i) Uc[i] = S->U[i * nc + c];
    rc = equilibrium_with(&S->g, S->C, S->A, Uc, S->tmpM, S->tmpF);
    if (rc) break;
    for (long k = 0; k < nv; ++k) S->f[k * nc + c] = S->tmpF[k];
  }
  double* lam = S->lam;
  if (!rc) {
    S->lam = lam_eff;
    rc = step_hofks(S);
    S->lam = lam;
  }
  for (long c = 0; !rc && !keep_raw && c < nc; ++c) {
    if (!(flags[c] != 0 && lam[c] != 1.0)) continue;
    for (int i = 0; i < nm; ++i) Uc[i] = S->U[i * nc + c];
    rc = equilibrium_with(&S->g, S->C, S->A, Uc, S->tmpM, S->tmpF);
    if (rc) break;
    for (long k = 0; k < nv; ++k) S->f[k * nc + c] = S->tmpF[k];
  }
  free(lam_eff);
  if (rc) return rc;
  S->n += 1;
  for (long c = 0; c < nc; ++c) {
    double rho, u[3], theta;
    for (int i = 0; i < nm; ++i) Uc[i] = S->U[i * nc + c];
    rc = primitives(S->g.d, Uc, &rho, u, &theta);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* Size of the departure from equilibrium at every cell:
 *   out[c] = log10(max(||f_c - E[U_c]||_1 / ||E[U_c]||_1, 1e-12)),
 * discrete L1 norms over the velocities (the dv^d factor cancels).  f is
 * nv x nc at cell positions, U is nm x nc. */
int orc_noneq(const orc_config* g, const double* f, const double* U, double* out) {
  int rc = check_config(g);
  if (rc) return rc;
  const int nm = g->d + 2;
  const long nc = ncells(g), nv = nvel(g);
  double* C = malloc(sizeof(double) * nm * nv);
  double* M = malloc(sizeof(double) * nv);
  double* E = malloc(sizeof(double) * nv);
  double A[MAXM * MAXM];
  if (!C || !M || !E) rc = ORC_ERR_OOM;
  if (!rc) rc = orc_matrices(g, C, A);
  for (long c = 0; !rc && c < nc; ++c) {
    double Uc[MAXM];
    for (int i = 0; i < nm; ++i) Uc[i] = U[i * nc + c];
    rc = equilibrium_with(g, C, A, Uc, M, E);
    if (rc) break;
    double num = 0.0, den = 0.0;
    for (long k = 0; k < nv; ++k) {
      num += fabs(f[k * nc + c] - E[k]);
      den += fabs(E[k]);
    }
    const double r = num / den;
    out[c] = log10(r > 1e-12 ? r : 1e-12);
  }
  free(C);
  free(M);
  free(E);
  return rc;
}

/* Ten regime features per cell (the inputs of the regime classifier):
 *   0 rho, 1 u_x, 2 u_y, 3 theta, 4 log10 tau,
 *   5 log10 K(tau sqrt(theta) |grad ln rho|),  6 log10 K(tau sqrt(theta) |grad ln theta|),
 *   7 log10 K(tau |div u|),  8 log10 K(tau |d u_x / dy|),  9 log10 K(tau |d u_y / dx|),
 * K(a) = max(a, 1e-12).  Derivatives are central differences over the two
 * neighbours along each direction (the boundary rule of that direction
 * supplies missing neighbours); u_y and the y-derivatives are 0 in 1D.
 * tau is per cell (nc values).  out[i*nc + c]. */
int orc_features(const orc_config* g, const double* U, const double* tau, double* out) {
  int rc = check_config(g);
  if (rc) return rc;
  const int d = g->d, nm = d + 2;
  const long nc = ncells(g);
  double* prim = malloc(sizeof(double) * 5 * nc); /* rho, u_x, u_y, u_z, theta */
  if (!prim) return ORC_ERR_OOM;
  for (long c = 0; c < nc; ++c) {
    double Uc[MAXM], rho, u[3], theta;
    for (int i = 0; i < nm; ++i) Uc[i] = U[i * nc + c];
    rc = primitives(d, Uc, &rho, u, &theta);
    if (rc) {
      free(prim);
      return rc;
    }
    prim[0 * nc + c] = rho;
    for (int i = 0; i < 3; ++i) prim[(1 + i) * nc + c] = u[i];
    prim[4 * nc + c] = theta;
  }
  const double h2 = 2.0 * g->dx;
  for (long c = 0; c < nc; ++c) {
    /* D[q][i]: central difference of quantity q along direction i, q = ln rho,
     * ln theta, u_x, u_y, u_z */
    double Dq[5][3] = {{0}};
    for (int i = 0; i < d; ++i) {
      const long cp = neighbour(g, c, i, +1), cm = neighbour(g, c, i, -1);
      Dq[0][i] = (log(prim[cp]) - log(prim[cm])) / h2;
      Dq[1][i] = (log(prim[4 * nc + cp]) - log(prim[4 * nc + cm])) / h2;
      for (int j = 0; j < 3; ++j)
        Dq[2 + j][i] = (prim[(1 + j) * nc + cp] - prim[(1 + j) * nc + cm]) / h2;
    }
    const double rho = prim[c], theta = prim[4 * nc + c], t = tau[c];
    double glr = 0.0, glt = 0.0, div = 0.0;
    for (int i = 0; i < d; ++i) {
      glr += Dq[0][i] * Dq[0][i];
      glt += Dq[1][i] * Dq[1][i];
      div += Dq[2 + i][i];
    }
    const double kn[5] = {t * sqrt(theta) * sqrt(glr), t * sqrt(theta) * sqrt(glt),
                          t * fabs(div), t * fabs(Dq[2][1]), t * fabs(Dq[3][0])};
    out[0 * nc + c] = rho;
    out[1 * nc + c] = prim[1 * nc + c];
    out[2 * nc + c] = prim[2 * nc + c];
    out[3 * nc + c] = theta;
    out[4 * nc + c] = log10(t);
    for (int j = 0; j < 5; ++j) out[(5 + j) * nc + c] = log10(kn[j] > 1e-12 ? kn[j] : 1e-12);
  }
  free(prim);
  return ORC_OK;
}

/* Deep copy of a scheme state (the one-step check runs on a copy). */
orc_state* orc_clone(const orc_state* S) {
  orc_state* T = orc_create(&S->g, S->lam, 0.0);
  if (!T) return NULL;
  /* orc_create took lambda as tau; overwrite with the exact lambdas */
  const size_t phase = sizeof(double) * (size_t)S->nc * (size_t)S->nv;
  const size_t mom = sizeof(double) * (size_t)S->nc * (size_t)S->nm;
  memcpy(T->lam, S->lam, sizeof(double) * S->nc);
  memcpy(T->lamh, S->lamh, sizeof(double) * S->nc);
  memcpy(T->f, S->f, phase);
  memcpy(T->U, S->U, mom);
  memcpy(T->UE, S->UE, mom);
  memcpy(T->UM, S->UM, mom);
  memcpy(T->Us, S->Us, mom);
  T->n = S->n;
  T->last_m = S->last_m;
  for (int i = 0; i < 3; ++i) T->alpha[i] = S->alpha[i];
  return T;
}

/* Replace the per-cell lambda = exp(-dt/tau) of a state (nc values). */
void orc_set_lambda(orc_state* S, const double* lam) {
  memcpy(S->lam, lam, sizeof(double) * S->nc);
}
