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
  return 0;
}
