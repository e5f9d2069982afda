/*
 * A plain C11 consumer of include/mera.h, built and run by
 * tests/test_abi_host.py: the header compiles as C, the library links from
 * C, and the host-only entry points answer as documented.  No device call.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mera.h"

#define CHECK(cond)                                              \
  do {                                                           \
    if (!(cond)) {                                               \
      fprintf(stderr, "line %d: check failed: %s\n", __LINE__, #cond); \
      return 1;                                                  \
    }                                                            \
  } while (0)

int main(void) {
  CHECK(strstr(mera_version(), "sm_103a") != NULL);

  size_t ws = 0;
  CHECK(mera_workspace_size(MERA_OP_ASCEND, 16, 16, MERA_PREC_BF16X3, &ws) == MERA_OK && ws > 0);
  CHECK(mera_workspace_size(MERA_OP_ASCEND, 0, 16, MERA_PREC_BF16X3, &ws) == MERA_EINVAL);
  CHECK(strlen(mera_last_error()) > 0);

  double fa = 0.0, fd = 0.0;
  CHECK(mera_flops(MERA_OP_ASCEND, 16, 16, &fa) == MERA_OK);
  CHECK(mera_flops(MERA_OP_DESCEND, 16, 16, &fd) == MERA_OK);
  CHECK(fa > 6.0e11 && fa < 6.4e11 && fa == fd); /* two diagrams of 4 chi^9 + 8 chi^8 + lower */

  double* h1 = malloc(4096 * sizeof(double));
  double shift = 0.0;
  CHECK(h1 != NULL);
  CHECK(mera_ising_h1(1.0, h1, &shift) == MERA_OK);
  double tr = 0.0, asym = 0.0;
  for (int i = 0; i < 64; ++i) {
    tr += h1[i * 64 + i];
    CHECK(h1[i * 64 + i] <= 1e-12); /* negative semidefinite: no positive diagonal entry */
    for (int j = 0; j < 64; ++j) asym = fmax(asym, fabs(h1[i * 64 + j] - h1[j * 64 + i]));
  }
  CHECK(shift > 0.0 && tr < 0.0 && asym == 0.0);
  free(h1);

  size_t len = 0;
  CHECK(mera_plan_json(MERA_OP_ENV_W, 8, 8, MERA_PREC_F64, NULL, 0, &len) == MERA_OK && len > 0);
  char* js = malloc(len + 1);
  CHECK(js != NULL);
  CHECK(mera_plan_json(MERA_OP_ENV_W, 8, 8, MERA_PREC_F64, js, len + 1, &len) == MERA_OK);
  CHECK(js[0] == '{' && js[len - 1] == '}' && strlen(js) == len);
  free(js);

  /* three MERAs of three layers: chi = 8, 16, 8 */
  const int cb[9] = {4, 8, 8, 4, 16, 16, 4, 8, 8};
  const int ct[9] = {8, 8, 8, 16, 16, 16, 8, 8, 8};
  size_t need[3];
  for (int i = 0; i < 3; ++i)
    CHECK(mera_sweep_workspace_size(3, cb + 3 * i, ct + 3 * i, MERA_PREC_BF16X3, &need[i]) == MERA_OK);
  int lane[3], n_lanes = 0;
  size_t lane_bytes[3];
  CHECK(mera_batch_lanes(3, 3, cb, ct, MERA_PREC_BF16X3, 20, need[1], 8, lane, &n_lanes, lane_bytes) == MERA_OK);
  CHECK(n_lanes == 1 && lane[0] == 0 && lane[1] == 0 && lane[2] == 0 && lane_bytes[0] == need[1]);
  CHECK(mera_batch_lanes(3, 3, cb, ct, MERA_PREC_BF16X3, 20, need[1] - 1, 8, lane, &n_lanes, lane_bytes) ==
        MERA_ENOMEM);

  int n = -1;
  CHECK(mera_autotune_reset() == MERA_OK);
  CHECK(mera_set_tile_width(MERA_PREC_BF16X3, 65536, 256, 4096, 1, 96) == MERA_EINVAL);
  CHECK(mera_set_tile_width(MERA_PREC_BF16X3, 65536, 256, 4096, 1, 128) == MERA_OK);
  long long rec[6];
  CHECK(mera_tile_widths(rec, 1, &n) == MERA_OK && n == 1);
  CHECK(rec[0] == MERA_PREC_BF16X3 && rec[1] == 65536 && rec[2] == 256 && rec[3] == 4096 && rec[4] == 1 &&
        rec[5] == 128);
  CHECK(mera_autotune_reset() == MERA_OK && mera_tile_widths(NULL, 0, &n) == MERA_OK && n == 0);

  puts("abi consumer ok");
  return 0;
}
