/* A plain C99 consumer of the C ABI: compiled against include/hps.h and linked with
 * libhps.so by tests/test_abi.py.  It needs no GPU: it checks the status messages, the
 * rejection of a null context and of bad sizes, and that context creation either succeeds
 * (a device is present) or reports HPS_ENODEV. */
#include <stdio.h>
#include <string.h>

#include "hps.h"

int main(void) {
  const int statuses[] = {HPS_OK, HPS_EINVAL, HPS_ENOMEM, HPS_ENOTBUILT, HPS_ENOTCONV,
                          HPS_ETIMEOUT, HPS_ECUDA, HPS_ENODEV, HPS_EUNSUPPORTED, HPS_ENUMERIC};
  size_t i;
  hps_ctx* ctx = NULL;
  int st;
  for (i = 0; i < sizeof statuses / sizeof statuses[0]; ++i) {
    const char* m = hps_strerror(statuses[i]);
    if (m == NULL || m[0] == '\0') {
      printf("empty message for status %d\n", statuses[i]);
      return 1;
    }
  }
  if (hps_mesh(NULL, 4, 4, 8) != HPS_EINVAL || hps_destroy(NULL) != HPS_OK) {
    printf("null context not rejected\n");
    return 2;
  }
  if (hps_create(NULL, 0, NULL) != HPS_EINVAL) {
    printf("null handle pointer not rejected\n");
    return 3;
  }
  st = hps_create(&ctx, 0, NULL);
  if (st == HPS_OK) {
    /* a device is present: a mesh that is not 2^k x 2^k is refused, a valid one accepted */
    long long n_skel = 0, n_bdry = 0, held = 0;
    int levels = 0;
    if (hps_mesh(ctx, 3, 3, 8) != HPS_EINVAL || hps_mesh(ctx, 4, 4, 8) != HPS_OK ||
        hps_sizes(ctx, &n_skel, &n_bdry, &levels, &held) != HPS_OK || n_skel != 2 * 24 * 7 ||
        n_bdry != 4 * 4 * 7 || levels != 4) {
      printf("mesh checks failed: %s\n", hps_last_error(ctx));
      hps_destroy(ctx);
      return 4;
    }
    hps_destroy(ctx);
    printf("device\n");
    return 0;
  }
  if (st != HPS_ENODEV || ctx != NULL) {
    printf("unexpected status %d without a device\n", st);
    return 5;
  }
  printf("no device\n");
  return 0;
}
