/* Prints the size and field offsets of every struct in include/ftgemm.h as
 * "struct.field offset" lines ("struct sizeof N" for the size), so the
 * Python binding's ctypes declarations can be compared with the C layout. */
#include <stddef.h>
#include <stdio.h>

#include "ftgemm.h"

#define F(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f))
#define SZ(T) printf("%s sizeof %zu\n", #T, sizeof(T))

int main(void) {
  SZ(ftgemm_loc);
  F(ftgemm_loc, row); F(ftgemm_loc, col); F(ftgemm_loc, tile); F(ftgemm_loc, kind); F(ftgemm_loc, delta);
  SZ(ftgemm_report);
  F(ftgemm_report, detected); F(ftgemm_report, corrected); F(ftgemm_report, checksum_only);
  F(ftgemm_report, unverifiable); F(ftgemm_report, flagged_rows); F(ftgemm_report, flagged_cols);
  F(ftgemm_report, recomputed); F(ftgemm_report, panel_detected); F(ftgemm_report, n_loc);
  F(ftgemm_report, cap); F(ftgemm_report, loc);
  SZ(ftgemm_flip);
  F(ftgemm_flip, row); F(ftgemm_flip, col); F(ftgemm_flip, kstep); F(ftgemm_flip, bit); F(ftgemm_flip, problem);
  SZ(ftgemm_inject);
  F(ftgemm_inject, mode); F(ftgemm_inject, pad); F(ftgemm_inject, seed); F(ftgemm_inject, count);
  F(ftgemm_inject, list); F(ftgemm_inject, n_list);
  SZ(ftgemm_flip_log);
  F(ftgemm_flip_log, row); F(ftgemm_flip_log, col); F(ftgemm_flip_log, kstep); F(ftgemm_flip_log, bit);
  F(ftgemm_flip_log, applied); F(ftgemm_flip_log, before); F(ftgemm_flip_log, after); F(ftgemm_flip_log, kfirst);
  F(ftgemm_flip_log, problem);
  return 0;
}
