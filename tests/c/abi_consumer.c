/* A plain C99 consumer of the library's C ABI: builds against the public
   header alone and exercises the host-side calls (no device work), checking
   the status codes the header documents. */
#include <stdio.h>
#include <string.h>

#include "qmckl_gpu.h"

#define EXPECT(call, want)                                                     \
  do {                                                                         \
    qk_status st_ = (call);                                                    \
    if (st_ != (want)) {                                                       \
      fprintf(stderr, "%s:%d: %s returned %d, expected %d\n", __FILE__,        \
              __LINE__, #call, (int)st_, (int)(want));                         \
      return 1;                                                                \
    }                                                                          \
  } while (0)

int main(void) {
  qk_context ctx = NULL;
  EXPECT(qk_context_create(&ctx), QK_SUCCESS);
  EXPECT(qk_context_destroy(NULL), QK_ERR_NULL_POINTER);
  EXPECT(qk_set_compute_mode(ctx, QK_BF16X3), QK_SUCCESS);
  EXPECT(qk_set_compute_mode(ctx, 7), QK_ERR_INVALID_ARG);
  EXPECT(qk_set_cutoff(ctx, 1e-10), QK_SUCCESS);

  /* one nucleus with an s shell (2 primitives) and a p shell (1 primitive) */
  const double charge[1] = {8.0};
  const double coord[3] = {0.0, 0.0, 0.0};
  const int64_t shell_nucleus[2] = {0, 0};
  const int32_t shell_ang_mom[2] = {0, 1};
  const int64_t shell_prim_num[2] = {2, 1};
  const double shell_factor[2] = {1.0, 1.0};
  const double exponent[3] = {5.0, 0.5, 1.2};
  const double coefficient[3] = {0.4, 0.6, 1.0};
  const double prim_factor[3] = {1.0, 1.0, 1.0};
  const double ao_factor[4] = {1.0, 1.0, 1.0, 1.0};
  const double C[2 * 4] = {1, 0, 0, 0, 0, 1, 1, 1};

  EXPECT(qk_set_ao_basis(ctx, 2, 3, shell_nucleus, shell_ang_mom, shell_prim_num,
                         shell_factor, exponent, coefficient, prim_factor, 4, ao_factor),
         QK_ERR_NOT_PROVIDED); /* nuclei first */
  EXPECT(qk_set_nucleus(ctx, 1, charge, coord), QK_SUCCESS);
  EXPECT(qk_set_ao_basis(ctx, 2, 3, shell_nucleus, shell_ang_mom, shell_prim_num,
                         shell_factor, exponent, coefficient, prim_factor, 3, ao_factor),
         QK_ERR_BAD_SIZE); /* ao_num does not match the shells (1 + 3) */
  EXPECT(qk_set_ao_basis(ctx, 2, 3, shell_nucleus, shell_ang_mom, shell_prim_num,
                         shell_factor, exponent, coefficient, prim_factor, 4, ao_factor),
         QK_SUCCESS);
  EXPECT(qk_set_mo_coefficient(ctx, 2, C), QK_SUCCESS);

  int64_t n = 0;
  EXPECT(qk_get_ao_num(ctx, &n), QK_SUCCESS);
  if (n != 4) return 2;
  EXPECT(qk_get_mo_num(ctx, &n), QK_SUCCESS);
  if (n != 2) return 3;

  const double pts[3] = {0.1, 0.2, 0.3};
  EXPECT(qk_set_points(ctx, 'N', 0, 1, pts), QK_ERR_BAD_SIZE);
  EXPECT(qk_set_points(ctx, 'X', 1, 1, pts), QK_ERR_INVALID_ARG);
  EXPECT(qk_set_points(ctx, 'N', 1, 1, NULL), QK_ERR_NULL_POINTER);

  char msg[256];
  EXPECT(qk_last_error(ctx, msg, (int64_t)sizeof msg), QK_SUCCESS);
  if (strlen(msg) == 0) return 4;

  EXPECT(qk_context_destroy(ctx), QK_SUCCESS);
  printf("ok\n");
  return 0;
}
