/* Plain C99 use of include/dg.h: the header compiles as C, the library links,
 * and the calls that need no GPU behave as documented (status codes, error
 * strings, NULL handling, argument validation before any device work). */
#include <stdio.h>
#include <string.h>
#include "dg.h"

static int fails = 0;
#define CHECK(cond)                                                    \
  do {                                                                 \
    if (!(cond)) {                                                     \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
      ++fails;                                                         \
    }                                                                  \
  } while (0)

int main(void) {
  CHECK(strcmp(dg_strerror(DG_OK), "ok") == 0);
  CHECK(strcmp(dg_strerror(DG_EMESH), "invalid mesh") == 0);
  dg_ctx* ctx = (dg_ctx*)0x1;
  CHECK(dg_mesh_setup(NULL, 2, DG_FP64, 1.0, 0, &ctx) == DG_EINVAL);
  CHECK(ctx == NULL);
  /* a one-element mesh whose only neighbour index is out of range */
  double nodes[8 * 3] = {0};
  int32_t nbr[6] = {-1, -1, -1, -1, -1, 5};
  int8_t nbr_face[6] = {0}, orient[6] = {0};
  dg_mesh_desc m = {1, 1, nodes, nbr, nbr_face, orient};
  CHECK(dg_mesh_setup(&m, 2, DG_FP64, 1.0, 0, &ctx) == DG_EMESH);
  CHECK(dg_last_error(NULL) != NULL && strlen(dg_last_error(NULL)) > 0);
  CHECK(dg_mesh_setup(&m, DG_KMAX + 1, DG_FP64, 1.0, 0, &ctx) == DG_EUNSUPPORTED);
  CHECK(dg_apply_operator(NULL, NULL, NULL, 0) == DG_EINVAL);
  CHECK(dg_get_state(NULL, NULL, NULL, 0) == DG_EINVAL);
  CHECK(dg_set_predictor_kernel(NULL, DG_PRED_AUTO) == DG_EINVAL);
  dg_destroy(NULL);
  if (fails == 0) printf("c abi ok\n");
  return fails == 0 ? 0 : 1;
}
