/*
 * riemann.c -- exact solution of the 1D Euler Riemann problem for an ideal
 * gas (the classical exact solver: pressure function of the two non-linear
 * waves, root found by bisection, then the similarity solution sampled at
 * x/t).  Used by the tests as an independent pin of the tau -> 0 limit of
 * HOFKS (the paper compares its 1D Sod results with Euler solvers in
 * Section 5.1).  TEST INFRASTRUCTURE ONLY.
 */
#include <math.h>

#include "dvm_oracle.h"

/* Velocity jump across the K wave as a function of the star pressure p:
 * a shock if p > pk (Rankine-Hugoniot), a rarefaction otherwise
 * (isentropic, Riemann invariant). */
static double wave_jump(double gamma, double p, double rk, double pk) {
  const double ck = sqrt(gamma * pk / rk);
  if (p > pk) {
    const double Ak = 2.0 / ((gamma + 1.0) * rk);
    const double Bk = (gamma - 1.0) / (gamma + 1.0) * pk;
    return (p - pk) * sqrt(Ak / (p + Bk));
  }
  return 2.0 * ck / (gamma - 1.0) *
         (pow(p / pk, (gamma - 1.0) / (2.0 * gamma)) - 1.0);
}

static void sample(double gamma, double rl, double ul, double pl, double rr,
                   double ur, double pr, double ps, double us, double xi,
                   double* r, double* u, double* p) {
  const double g1 = (gamma - 1.0) / (gamma + 1.0);
  if (xi <= us) { /* left of the contact */
    const double cl = sqrt(gamma * pl / rl);
    if (ps > pl) {
      const double sl =
          ul - cl * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl +
                         (gamma - 1.0) / (2.0 * gamma));
      if (xi <= sl) {
        *r = rl; *u = ul; *p = pl;
      } else {
        *r = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0);
        *u = us; *p = ps;
      }
    } else {
      const double csl = cl * pow(ps / pl, (gamma - 1.0) / (2.0 * gamma));
      const double head = ul - cl, tail = us - csl;
      if (xi <= head) {
        *r = rl; *u = ul; *p = pl;
      } else if (xi >= tail) {
        *r = rl * pow(ps / pl, 1.0 / gamma);
        *u = us; *p = ps;
      } else {
        const double t = 2.0 / (gamma + 1.0) +
                         (gamma - 1.0) / ((gamma + 1.0) * cl) * (ul - xi);
        *r = rl * pow(t, 2.0 / (gamma - 1.0));
        *u = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * ul + xi);
        *p = pl * pow(t, 2.0 * gamma / (gamma - 1.0));
      }
    }
  } else { /* right of the contact */
    const double cr = sqrt(gamma * pr / rr);
    if (ps > pr) {
      const double sr =
          ur + cr * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr +
                         (gamma - 1.0) / (2.0 * gamma));
      if (xi >= sr) {
        *r = rr; *u = ur; *p = pr;
      } else {
        *r = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0);
        *u = us; *p = ps;
      }
    } else {
      const double csr = cr * pow(ps / pr, (gamma - 1.0) / (2.0 * gamma));
      const double head = ur + cr, tail = us + csr;
      if (xi >= head) {
        *r = rr; *u = ur; *p = pr;
      } else if (xi <= tail) {
        *r = rr * pow(ps / pr, 1.0 / gamma);
        *u = us; *p = ps;
      } else {
        const double t = 2.0 / (gamma + 1.0) -
                         (gamma - 1.0) / ((gamma + 1.0) * cr) * (ur - xi);
        *r = rr * pow(t, 2.0 / (gamma - 1.0));
        *u = 2.0 / (gamma + 1.0) * (-cr + 0.5 * (gamma - 1.0) * ur + xi);
        *p = pr * pow(t, 2.0 * gamma / (gamma - 1.0));
      }
    }
  }
}

int orc_riemann_exact(double gamma, double rl, double ul, double pl,
                      double rr, double ur, double pr, const double* xi,
                      int npts, double* rho, double* u, double* pres,
                      double* pstar, double* ustar) {
  if (!(rl > 0 && rr > 0 && pl > 0 && pr > 0 && gamma > 1)) return ORC_ERR_ARG;
  const double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
  /* no vacuum: the pressure-positivity condition of the exact solver */
  if (2.0 * (cl + cr) / (gamma - 1.0) <= ur - ul) return ORC_ERR_ARG;
  /* g(p) = f_L(p) + f_R(p) + (u_R - u_L) is increasing in p */
  double lo = 0.0, hi = fmax(pl, pr);
  while (wave_jump(gamma, hi, rl, pl) + wave_jump(gamma, hi, rr, pr) + (ur - ul) < 0.0)
    hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    const double gval =
        wave_jump(gamma, mid, rl, pl) + wave_jump(gamma, mid, rr, pr) + (ur - ul);
    if (gval < 0.0) lo = mid; else hi = mid;
  }
  const double ps = 0.5 * (lo + hi);
  const double us = 0.5 * (ul + ur) +
                    0.5 * (wave_jump(gamma, ps, rr, pr) - wave_jump(gamma, ps, rl, pl));
  for (int i = 0; i < npts; ++i)
    sample(gamma, rl, ul, pl, rr, ur, pr, ps, us, xi[i], &rho[i], &u[i], &pres[i]);
  if (pstar) *pstar = ps;
  if (ustar) *ustar = us;
  return ORC_OK;
}
