/* Plain-C use of include/rqrcp.h: compiled as C99 with warnings as errors and
 * linked against librqrcp.so by the CPU tests.  Every entry point is taken as
 * a typed function pointer (the declarations are valid C), and the calls that
 * need no GPU run: the posterior CDF, the padding helper and the tile search
 * with a C cost function.  Test infrastructure only. */
#include <stdio.h>

#include "rqrcp.h"

static int bowl(void* user, const rq_batch_tiles* t, double* ms) {
  int* calls = (int*)user;
  int dm = t->skinny_m - 64, dn = t->skinny_n - 16;
  ++*calls;
  *ms = 1.0 + (dm < 0 ? -dm : dm) / 16.0 + (dn < 0 ? -dn : dn) / 16.0;
  return 0;
}

typedef void (*fn_t)(void);

int main(void) {
  fn_t fns[] = {
      (fn_t)rq_create,         (fn_t)rq_destroy,       (fn_t)rq_workspace_size, (fn_t)rq_set_workspace,
      (fn_t)rq_last_error,     (fn_t)rq_launch_count,  (fn_t)rq_profile_enable, (fn_t)rq_profile_read,
      (fn_t)rq_rqrcp,          (fn_t)rq_rqrcp_noalloc, (fn_t)rq_gaussian,       (fn_t)rq_rsrqrcp,
      (fn_t)rq_latent_cdf,     (fn_t)rq_padding,       (fn_t)rq_qr,             (fn_t)rq_trqrcp,
      (fn_t)rq_tuxv,           (fn_t)rq_tuxv_iter,     (fn_t)rq_tuxv_batched,   (fn_t)rq_gemm_bf16,
      (fn_t)rq_set_batch_tiles, (fn_t)rq_get_batch_tiles, (fn_t)rq_tiles_search, (fn_t)rq_tune_batched,
      (fn_t)rq_selftest_wait_timeout, (fn_t)rq_gemm_f64, (fn_t)rq_copy};
  unsigned i, missing = 0;
  double prob = -1.0;
  int p = -1, rc, calls = 0;
  rq_batch_tiles best;
  double best_ms = 0.0;
  for (i = 0; i < sizeof fns / sizeof fns[0]; ++i) missing += fns[i] == NULL;
  rc = rq_latent_cdf(4, 0.125, &prob);
  printf("entry_points %u missing %u\n", (unsigned)(sizeof fns / sizeof fns[0]), missing);
  printf("latent_cdf %d %.6f\n", rc, prob);
  rc = rq_padding(0.125, 0.01, &p);
  printf("padding %d %d\n", rc, p);
  rc = rq_tiles_search(bowl, &calls, NULL, 3, &best, &best_ms);
  printf("tiles_search %d %d %d %.3f %d\n", rc, best.skinny_m, best.skinny_n, best_ms, calls);
  printf("destroy_null %d\n", rq_destroy(NULL));
  return 0;
}
