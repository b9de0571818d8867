/* Compiles include/hsgen.h as plain C11 and calls the entry points that need
 * no GPU: default options, argument checks on NULL, the error text of a NULL
 * context. Prints "ok" and exits 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "hsgen.h"

#define CHECK(c)                                             \
  do {                                                       \
    if (!(c)) {                                              \
      fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
      return 1;                                              \
    }                                                        \
  } while (0)

int main(void) {
  hsgen_options o;
  memset(&o, 0xff, sizeof(o));
  hsgen_default_options(&o);
  CHECK(o.precision == HSGEN_FP64);
  CHECK(o.uplo == 'U');
  CHECK(o.s_form == HSGEN_S_CONTRACTION);
  CHECK(o.target_rel_err == 1e-12);
  CHECK(o.wait_timeout_ns > 0);
  CHECK(hsgen_create(NULL, 0, NULL) == HSGEN_EINVAL);
  CHECK(hsgen_build_HS(NULL, 1, NULL, NULL, NULL, 1, NULL) == HSGEN_EINVAL);
  CHECK(hsgen_reduce_generalized(NULL, 1, NULL, NULL, 1, NULL) == HSGEN_EINVAL);
  CHECK(hsgen_get_stats(NULL, NULL) == HSGEN_EINVAL);
  CHECK(strcmp(hsgen_last_error(NULL), "null context") == 0);
  hsgen_destroy(NULL);
  printf("ok\n");
  return 0;
}
