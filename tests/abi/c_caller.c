/* A plain C caller of libftgemm: compiles against include/ftgemm.h as C11
 * with warnings as errors, links against the shared library, and exercises
 * the host-only paths (argument codes, the K-split query, error strings,
 * injection settings) that need no GPU.  Prints one line per check and
 * exits non-zero on the first mismatch. */
#include <stdio.h>
#include <string.h>

#include "ftgemm.h"

static int fails = 0;

static void expect(const char *what, long long got, long long want) {
  printf("%s: %lld (want %lld)\n", what, got, want);
  if (got != want) ++fails;
}

int main(void) {
  /* argument codes, BLAS numbering, before any device work */
  expect("ftgemm_d bad transA", ftgemm_d('X', 'N', 2, 2, 2, 1.0, NULL, 2, NULL, 2, 0.0, NULL, 2, NULL, NULL), -1);
  expect("ftgemm_d bad lda", ftgemm_d('N', 'N', 3, 2, 2, 1.0, NULL, 2, NULL, 2, 0.0, NULL, 3, NULL, NULL), -8);
  expect("ftgemm_d_noft bad ldc", ftgemm_d_noft('N', 'N', 3, 2, 2, 1.0, NULL, 3, NULL, 2, 0.0, NULL, 2, NULL), -13);
  expect("ftgemm_d_split bad nslices",
         ftgemm_d_split('N', 'N', 4, 4, 4, 1.0, NULL, 4, NULL, 4, 0.0, NULL, 4, 16, 0, NULL, NULL), -14);
  expect("ftgemm_encode_operands bad ldb",
         ftgemm_encode_operands('N', 'N', 2, 2, 3, NULL, 2, NULL, 2, NULL, NULL, NULL, NULL, NULL, NULL, NULL), -9);
  expect("ftgemm_batched count < 0",
         ftgemm_batched(-1, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL),
         FTGEMM_ERR_BATCH);

  /* an empty output is a quick return with a zeroed report */
  ftgemm_loc locs[4];
  ftgemm_report rep;
  memset(&rep, 0x7f, sizeof(rep));
  rep.cap = 4;
  rep.loc = locs;
  expect("ftgemm_d M = 0", ftgemm_d('N', 'N', 0, 5, 5, 1.0, NULL, 1, NULL, 5, 0.0, NULL, 1, &rep, NULL), 0);
  expect("report zeroed", rep.detected + rep.corrected + rep.n_loc, 0);

  /* the K-split plan, host only */
  int splits = 0;
  int64_t first = -1;
  expect("query 4096^3", ftgemm_query_ksplit(4096, 4096, 4096, 152, &splits, &first), 0);
  expect("  splits", splits, 4);
  expect("  first split tile", first, 912);

  /* injection settings and error strings */
  ftgemm_flip f = {1, 2, 0, 5, 0};
  ftgemm_inject cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.mode = 2;
  cfg.list = &f;
  cfg.n_list = 1;
  expect("set explicit injection", ftgemm_set_injection(&cfg), 0);
  expect("clear injection", ftgemm_set_injection(NULL), 0);
  expect("strerror(0) is success", strcmp(ftgemm_strerror(0), "success"), 0);
  expect("launches", ftgemm_launch_count(), 0);
  return fails ? 1 : 0;
}
