/* A plain C99 client of include/rsvd.h: the header compiles as C, the library
 * links, and the calls that need no GPU (version, size queries, error strings,
 * argument checks) answer as documented. Exit status 0 = every check held; a
 * failing check prints its line. */
#include <stdio.h>
#include <string.h>

#include "rsvd.h"

static int failed = 0;
#define CHECK(cond)                                           \
  do {                                                        \
    if (!(cond)) {                                            \
      fprintf(stderr, "check failed (line %d): %s\n", __LINE__, #cond); \
      failed = 1;                                             \
    }                                                         \
  } while (0)

int main(void) {
  const double k[4] = {1.0, 2.0, 3.0, 4.0};
  void* dummy = (void*)(size_t)256; /* never dereferenced: every call below fails its argument check */
  float* fdummy = (float*)dummy;
  int32_t* idummy = (int32_t*)dummy;

  CHECK(rsvd_abi_version() == RSVD_ABI_VERSION);
  CHECK(rsvd_strerror(RSVD_OK) != NULL && strlen(rsvd_strerror(RSVD_EINVAL)) > 0);
  CHECK(strcmp(rsvd_strerror(RSVD_EINVAL), rsvd_strerror(RSVD_EUNSUPPORTED)) != 0);

  /* FP32 compressed rings: N x T rows of H components at Q/2 complex slots */
  CHECK(rsvd_compressed_bytes(4, 9, 12, 256, RSVD_FP32) == (size_t)4 * 9 * 12 * 128 * 8);
  CHECK(rsvd_compressed_bytes(0, 9, 12, 256, RSVD_FP32) == 0);
  /* the split form holds two bf16 planes: twice the single-pass form */
  CHECK(rsvd_compressed_bytes(4, 9, 12, 256, RSVD_BF16X3) == 2 * rsvd_compressed_bytes(4, 9, 12, 256, RSVD_BF16));
  /* the scaled half split: two fp16 planes, then one float factor per row (16-byte padded) */
  CHECK(rsvd_compressed_bytes(4, 9, 12, 256, RSVD_FP16X3) ==
        rsvd_compressed_bytes(4, 9, 12, 256, RSVD_BF16X3) + (size_t)((4 * 9 * 4 + 15) / 16 * 16));
  CHECK(rsvd_build_workspace_bytes(64, 256, 1024) > 0);
  CHECK(rsvd_align_host_workspace_bytes(64, 256, 12, 9, 1024, 0, RSVD_FP32, 0) == 0); /* chunk 0 */

  /* argument errors: nothing is enqueued, so no GPU is needed */
  CHECK(rsvd_align_best(NULL, 1, 1, dummy, 1, 8, 256, RSVD_FP32, 1.0f, fdummy, idummy, NULL, NULL) == RSVD_EINVAL);
  CHECK(rsvd_align_best(dummy, 0, 1, dummy, 1, 8, 256, RSVD_FP32, 1.0f, fdummy, idummy, NULL, NULL) == RSVD_EINVAL);
  CHECK(rsvd_align_best(dummy, 1, 1, dummy, 1, 8, 256, RSVD_FP32, 0.0f, fdummy, idummy, fdummy, NULL) == RSVD_EINVAL);
  CHECK(rsvd_align_scores(dummy, 1, 1, dummy, 1, 8, 48, RSVD_FP32, fdummy, NULL) == RSVD_EUNSUPPORTED);
  CHECK(rsvd_compress(4, 16, k, k, (const double*)dummy, 5, dummy, 1, NULL, 1, RSVD_FP32, dummy, NULL) ==
        RSVD_EINVAL); /* H > R */
  CHECK(rsvd_build_radial_svd(4, 16, k, dummy, 3, 2, (double*)dummy, (double*)dummy, NULL, 0, NULL) ==
        RSVD_EWORKSPACE);

  if (!failed) printf("c abi ok\n");
  return failed;
}
