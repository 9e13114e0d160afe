/* Compiled by tests/test_abi.py as plain C99 against include/tsfcde.h and linked to
 * libtsfcde.so: the header is valid C, and the calls that need no device behave as declared. */
#include <stdio.h>
#include <string.h>

#include "tsfcde.h"

static double coef(double t, void *user) {
  (void)t;
  (void)user;
  return 1.0;
}
static void field(double t, const double *x, double *out, int64_t n, void *user) {
  (void)t;
  (void)user;
  for (int64_t i = 0; i < n; ++i) out[i] = x[i] * (1.0 - x[i]);
}

int main(void) {
  tsfcde_options opt;
  tsfcde_default_options(&opt);
  if (opt.precision != TSFCDE_FP64 || opt.preconditioner != TSFCDE_PRECOND_STRANG ||
      opt.tol != 1e-12 || opt.algorithm != TSFCDE_ALG_IDS || opt.inner_tol != 1e-3) {
    fprintf(stderr, "unexpected defaults\n");
    return 1;
  }
  if (strcmp(tsfcde_strerror(TSFCDE_OK), "ok") != 0 || strstr(tsfcde_version(), "sm_103a") == NULL) {
    fprintf(stderr, "strerror/version\n");
    return 2;
  }
  tsfcde_ctx *ctx = (tsfcde_ctx *)0x1;
  /* alpha out of (0, 1]: rejected before any device call, *out cleared */
  int st = tsfcde_setup(&ctx, 0.0, 1.0, 1.0, 15, 4, 1.5, 1.5, coef, coef, coef, field, NULL, NULL, &opt);
  if (st != TSFCDE_E_INVALID_ARG || ctx != NULL) {
    fprintf(stderr, "setup check %d\n", st);
    return 3;
  }
  opt.algorithm = 9;
  st = tsfcde_setup(&ctx, 0.0, 1.0, 1.0, 15, 4, 0.5, 1.5, coef, coef, coef, field, NULL, NULL, &opt);
  if (st != TSFCDE_E_INVALID_ARG) return 4;
  tsfcde_free(NULL);       /* NULL is allowed */
  tsfcde_batch_free(NULL);
  if (tsfcde_step(NULL, 1, NULL) != TSFCDE_E_INVALID_ARG) return 5;
  if (tsfcde_batch_step(NULL, 1, NULL) != TSFCDE_E_INVALID_ARG) return 6;
  {
    double u[15];
    int64_t lev = 0;
    if (tsfcde_get_level(NULL, 0, u) != TSFCDE_E_INVALID_ARG) return 7;
    if (tsfcde_level(NULL, &lev) != TSFCDE_E_INVALID_ARG) return 8;
    if (tsfcde_get_weights(NULL, u, u) != TSFCDE_E_INVALID_ARG) return 9;
    if (tsfcde_batch_get_level(NULL, 0, 0, u) != TSFCDE_E_INVALID_ARG) return 10;
    if (tsfcde_batch_level(NULL, &lev) != TSFCDE_E_INVALID_ARG) return 11;
  }
  /* the separable source is given as callbacks the library samples on its own mesh */
  {
    tsfcde_field_fn space[1] = {field};
    tsfcde_coef_fn time[1] = {coef};
    tsfcde_default_options(&opt);
    opt.source_rank = 1;
    opt.source_space = space;
    opt.source_time = time;
    opt.test_inject = TSFCDE_INJECT_NONE;
    /* a separable source and an f callback together: rejected */
    st = tsfcde_setup(&ctx, 0.0, 1.0, 1.0, 15, 4, 0.5, 1.5, coef, coef, coef, field, field, NULL, &opt);
    if (st != TSFCDE_E_INVALID_ARG) return 12;
  }
  printf("c abi ok\n");
  return 0;
}
