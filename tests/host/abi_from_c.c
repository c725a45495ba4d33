/* Test infrastructure: include/tcurve.h compiled as C11 and libtcurve.so
 * linked into a plain C program, calling the entry points that need no GPU
 * (versions, statuses, argument checks, the Rohlin-Viro printer).  Exit
 * status 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "tcurve.h"

static int failures = 0;
#define CHECK(c)                                       \
  do {                                                 \
    if (!(c)) {                                        \
      printf("FAILED %s (line %d)\n", #c, __LINE__);   \
      ++failures;                                      \
    }                                                  \
  } while (0)

int main(void) {
  char buf[64];
  CHECK(ts_max_degree() == 16);
  CHECK(strncmp(ts_status_str(TS_EOVERFLOW), "TS_EOVERFLOW", 12) == 0);
  CHECK(strncmp(ts_status_str(-1), "unknown", 7) == 0);

  /* <1<1> + 2>: bits 11001010 below the sentinel (code 458, d = 6) */
  uint64_t code = 458;
  CHECK(ts_scheme_string(6, &code, 1, buf, sizeof buf) == TS_OK && strcmp(buf, "<1<1> + 2>") == 0);
  code = 1;
  CHECK(ts_scheme_string(7, &code, 1, buf, sizeof buf) == TS_OK && strcmp(buf, "<J>") == 0);
  code = 0; /* never a valid code */
  CHECK(ts_scheme_string(6, &code, 1, buf, sizeof buf) == TS_EINVAL);

  /* argument checks answer before any device work */
  ts_tri *tri = NULL;
  const int32_t edges[4] = {0, 0, 1, 0};
  CHECK(ts_load_triangulation(0, edges, 1, &tri) == TS_EINVAL && tri == NULL);
  CHECK(ts_load_triangulation(17, edges, 1, &tri) == TS_EUNSUPPORTED);
  CHECK(ts_load_triangulation(3, edges, 1, NULL) == TS_EINVAL);
  CHECK(ts_load_triangulation(3, edges, 1, &tri) == TS_ENOTTRI);
  ts_hist *h = NULL;
  CHECK(ts_hist_create(0, 1, &h) == TS_EINVAL);
  CHECK(ts_hist_create(16, 5, &h) == TS_EINVAL);
  CHECK(ts_real_schemes(NULL, NULL, 0, NULL, NULL) == TS_EINVAL);
  CHECK(ts_enumerate(NULL, 0, 1, 0, NULL, NULL) == TS_EINVAL);
  CHECK(ts_selftest_wait(0, NULL) == TS_EINVAL);
  CHECK(ts_batch_create(0, NULL, NULL, NULL, NULL, 16, NULL) == TS_EINVAL);
  CHECK(ts_sign_words(NULL) == 0 && ts_code_words(NULL) == 0);
  ts_free_triangulation(NULL);
  ts_hist_free(NULL);
  ts_batch_free(NULL);

  printf("C ABI checks: %d failed\n", failures);
  return failures != 0;
}
