/* A plain C99 caller of the library's C ABI (include/dvm.h), compiled and run by
 * tests/test_abi.py without a GPU: it fills a dvm_config the way a C program would
 * and calls the host-only entry point dvm_workspace_bytes.  Prints one line per
 * case: status and bytes. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "dvm.h"

static dvm_config quadrant(int n, int nv, int precision) {
  dvm_config c;
  memset(&c, 0, sizeof c);
  c.grid.dim = 2;
  c.grid.nx[0] = c.grid.nx[1] = n;
  c.grid.nx[2] = 1;
  c.grid.dx = 1.0 / n;
  c.vel.n[0] = c.vel.n[1] = nv;
  c.vel.n[2] = 1;
  c.vel.kmin[0] = c.vel.kmin[1] = -nv / 2;
  c.vel.dv = 0.4;
  c.vel.shift_den = 1;
  c.tau = 1e-3;
  c.tau_field = NULL;
  c.bc[0][0] = c.bc[0][1] = c.bc[1][0] = c.bc[1][1] = DVM_BC_PERIODIC;
  c.bc[2][0] = c.bc[2][1] = DVM_BC_PERIODIC;
  c.scheme = DVM_HOFKS;
  c.precision = precision;
  return c;
}

int main(void) {
  size_t bytes = 0;
  dvm_config c = quadrant(64, 32, DVM_F32);
  int rc = dvm_workspace_bytes(&c, &bytes);
  printf("f32 %d %zu\n", rc, bytes);
  c = quadrant(64, 32, DVM_F64);
  rc = dvm_workspace_bytes(&c, &bytes);
  printf("f64 %d %zu\n", rc, bytes);
  c = quadrant(64, 32, DVM_F32);
  c.grid.dim = 4;
  bytes = 0;
  rc = dvm_workspace_bytes(&c, &bytes);
  printf("bad_dim %d %zu\n", rc, bytes);
  c = quadrant(64, 32, DVM_F32);
  c.tau = INFINITY;
  rc = dvm_workspace_bytes(&c, &bytes);
  printf("tau_inf %d %zu\n", rc, bytes);
  rc = dvm_workspace_bytes(NULL, &bytes);
  printf("null %d\n", rc);

  /* degenerate and invalid configurations: each must give DVM_ERR_ARG */
  c = quadrant(64, 32, DVM_F32); c.grid.nx[0] = 0;
  printf("bad_empty_grid %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.vel.n[1] = 0;
  printf("bad_no_velocities %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.grid.dx = 0.0;
  printf("bad_dx %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.vel.dv = -0.4;
  printf("bad_dv %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.vel.shift_den = 0;
  printf("bad_shift_den %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.tau = -1.0;
  printf("bad_tau %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.tau = NAN;
  printf("bad_tau_nan %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.bc[1][1] = DVM_BC_OUTFLOW;
  printf("bad_faces %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.scheme = 7;
  printf("bad_scheme %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.precision = 9;
  printf("bad_precision %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(8, 258, DVM_F32);
  printf("bad_too_many_velocities %d\n", dvm_workspace_bytes(&c, &bytes));
  c = quadrant(64, 32, DVM_F32); c.grid.nx[2] = 2;
  printf("bad_unused_dimension %d\n", dvm_workspace_bytes(&c, &bytes));
  /* the largest velocity grid per dimension is accepted */
  c = quadrant(8, 256, DVM_F32);
  printf("max_velocities %d\n", dvm_workspace_bytes(&c, &bytes));
  return 0;
}
