/* Plain-C client of the library's C ABI (include/ffeq.h, include/ffeq_batch.h):
 * compiled as C11 and linked against libffeq.so by tests/test_abi.py.  It makes
 * only host-side calls (plan validation, sizes, status strings), so it runs on
 * a machine without a GPU; it prints "ok" and exits 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "ffeq.h"
#include "ffeq_batch.h"

static int fails = 0;
#define CHECK(cond)                                              \
  do {                                                           \
    if (!(cond)) {                                               \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
      ++fails;                                                   \
    }                                                            \
  } while (0)

int main(void) {
  ffeq_problem p;
  memset(&p, 0, sizeof p);
  p.B = 256; p.U = 16; p.C = 8; p.n_sc = 1200; p.n_sym = 14;
  p.arch = FFEQ_FD; p.precision = FFEQ_BF16X3; p.estimate = FFEQ_UNBIASED; p.llr_bits = 4;

  ffeq_plan* plan = NULL;
  CHECK(ffeq_plan_create(&plan, &p) == FFEQ_OK && plan != NULL);
  size_t ws = 0;
  CHECK(ffeq_workspace_size(plan, &ws) == FFEQ_OK);
  CHECK(ws == (size_t)1200 * 8 * (16 + 14) * 16 * 8);
  size_t wopt = 0;
  CHECK(ffeq_fd_optimal_workspace_size(plan, &wopt) == FFEQ_OK && wopt > ws);
  size_t staging = 0;
  CHECK(ffeq_host_staging_size(plan, &staging) == FFEQ_OK && staging > ws);
  ffeq_plan_destroy(plan);

  /* Every equalizer of the problem statement; LAMA needs its iterations and the LLR constellation. */
  p.equalizer = FFEQ_MRC;
  CHECK(ffeq_plan_create(&plan, &p) == FFEQ_OK);
  ffeq_plan_destroy(plan);
  p.equalizer = FFEQ_LAMA;
  CHECK(ffeq_plan_create(&plan, &p) == FFEQ_ERR_INVALID_ARG);   /* lama_iters = 0 */
  p.lama_iters = 8;
  CHECK(ffeq_plan_create(&plan, &p) == FFEQ_OK);
  ffeq_plan_destroy(plan);

  /* Unequal clusters through the same ABI. */
  int sizes[8] = {16, 48, 32, 24, 40, 32, 40, 24};
  p.equalizer = FFEQ_LMMSE; p.lama_iters = 0;
  CHECK(ffeq_plan_create_clusters(&plan, &p, sizes) == FFEQ_OK);
  ffeq_plan_destroy(plan);
  sizes[0] = 17;
  CHECK(ffeq_plan_create_clusters(&plan, &p, sizes) == FFEQ_ERR_INVALID_ARG);

  /* Validation happens before any device work. */
  p.U = 33;
  CHECK(ffeq_plan_create(&plan, &p) == FFEQ_ERR_UNSUPPORTED);
  CHECK(ffeq_plan_create(NULL, &p) != FFEQ_OK);
  CHECK(strcmp(ffeq_status_string(FFEQ_OK), "ok") == 0);
  CHECK(ffeq_version() >= 100);
  ffeq_plan_destroy(NULL);

  if (fails) return 1;
  printf("ok\n");
  return 0;
}
