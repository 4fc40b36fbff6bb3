/* A plain C11 caller of the library: it includes both public headers, links
 * libsp_gb300.so and calls the entry points that need no GPU.  It checks that
 * the headers are valid C, that the struct layouts a C compiler gives agree with
 * the library's (sp_abi_size), the default options, the nested-dissection level
 * sizes of the 2D 512^2, b = 16 grid against k = (B-1)^2 - 4 (B/2-1)^2,
 * m = k + (B+1)^2 - (B-1)^2 (root: k = m = n^2 - 4 (n/2-1)^2), the argument
 * checks of sp_setup (rejected before any device call) and the status strings.
 * Prints "c abi ok" and returns 0 on success. */
#include <stdio.h>
#include <string.h>

#include "sp.h"
#include "sp_fno.h"

static int fails = 0;
#define CHECK(c)                                                  \
  do {                                                            \
    if (!(c)) {                                                   \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #c); \
      ++fails;                                                    \
    }                                                             \
  } while (0)

int main(void) {
  sp_opts o;
  sp_ctx *ctx = NULL;
  int nl = 0, nf[16], k[16], m[16], l;
  const int n = 512, b = 16;

  CHECK(sp_abi_size(0) == sizeof(sp_opts));
  CHECK(sp_abi_size(1) == sizeof(sp_info));
  CHECK(sp_abi_size(2) == 0);

  memset(&o, 0xff, sizeof o);
  sp_default_opts(&o);
  CHECK(o.maxit == 500 && o.restart == 200 && o.tol == 1e-8 && o.device == 0);
  CHECK(o.host_threads == 0 && o.max_rhs == 1 && o.setup_route == 0 && o.stencil == 0);

  CHECK(sp_front_sizes(2, n, b, 16, &nl, nf, k, m) == SP_OK);
  CHECK(nl == 6);
  for (l = 0; l < nl && l < 16; ++l) {
    const int B = b << l;
    const int kk = l + 1 < nl ? (B - 1) * (B - 1) - 4 * (B / 2 - 1) * (B / 2 - 1)
                              : n * n - 4 * (n / 2 - 1) * (n / 2 - 1);
    const int mm = l + 1 < nl ? kk + (B + 1) * (B + 1) - (B - 1) * (B - 1) : kk;
    const int ff = l + 1 < nl ? (n / B) * (n / B) : 1;
    if (l == 0) { /* leaf boxes eliminate all (b-1)^2 interior points */
      CHECK(k[0] == (b - 1) * (b - 1) && m[0] == (b + 1) * (b + 1) && nf[0] == ff);
    } else {
      CHECK(k[l] == kk && m[l] == mm && nf[l] == ff);
    }
  }
  CHECK(sp_front_sizes(2, 500, 16, 16, &nl, nf, k, m) == SP_ERR_ARG); /* n/b not 2^L */

  CHECK(sp_setup(4, 64, 4, 100.0, SP_PREC_FP64, NULL, NULL, &ctx) == SP_ERR_ARG);
  CHECK(ctx == NULL);
  CHECK(sp_setup(2, 64, 5, 100.0, SP_PREC_FP64, NULL, NULL, &ctx) == SP_ERR_ARG);
  CHECK(sp_setup(2, 64, 4, 100.0, SP_PREC_FP64, NULL, NULL, NULL) == SP_ERR_ARG);
  /* s = 4 pi^2 |k|^2 for k = (1, 0): resonant */
  CHECK(sp_setup(2, 64, 4, 39.47841760435743, SP_PREC_FP64, NULL, NULL, &ctx) ==
        SP_ERR_RESONANT);

  CHECK(strcmp(sp_status_str(SP_OK), "ok") == 0);
  CHECK(strcmp(sp_status_str((sp_status)99), "unknown status") == 0);
  sp_destroy(NULL);

  if (fails) return 1;
  printf("c abi ok\n");
  return 0;
}
