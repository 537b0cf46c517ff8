/* C99 client of the boundary: include/nk.h must compile as plain C, the
 * library must link from C, and the host-only entry points must answer
 * without a GPU (status strings; the per-image self-variance count of an
 * architecture, one entry per pixel of every activation layer).  Every
 * declared entry point is also taken by address, so a C/C++ signature
 * mismatch in the header fails to compile or link.  Prints "ok". */
#include <stdio.h>
#include <string.h>

#include "nk.h"
#include "nk_probe.h"

static int fails = 0;
#define CHECK(cond)                                   \
  do {                                                \
    if (!(cond)) {                                    \
      printf("FAIL line %d: %s\n", __LINE__, #cond); \
      ++fails;                                        \
    }                                                 \
  } while (0)

int main(void) {
  /* every entry point, by address */
  const void* fns[] = {
      (const void*)&nk_create,         (const void*)&nk_destroy,          (const void*)&nk_status_string,
      (const void*)&nk_last_error,     (const void*)&nk_sync_status,      (const void*)&nk_q_size,
      (const void*)&nk_launch_count,   (const void*)&nk_last_lambda,      (const void*)&nk_self_diag,
      (const void*)&nk_block,          (const void*)&nk_block_backward,   (const void*)&nk_fc_block,
      (const void*)&nk_autotune,       (const void*)&nk_autotune_set,     (const void*)&nk_block_fused_noalloc,
      (const void*)&nk_block_ntk,      (const void*)&nk_block_queue,      (const void*)&nk_pcg_set_rank, (const void*)&nk_pcg_set_warm_start,
      (const void*)&nk_set_wait_limit, (const void*)&nk_probe,
      (const void*)&nk_pcg_solve,
  };
  for (size_t i = 0; i < sizeof(fns) / sizeof(fns[0]); ++i) CHECK(fns[i] != NULL);

  for (int s = 0; s <= 7; ++s) {
    const char* m = nk_status_string((nk_status)s);
    CHECK(m != NULL && strlen(m) > 0);
  }
  nk_arch a;
  memset(&a, 0, sizeof(a));
  a.n_stages = 3;
  a.convs[0] = 2;
  a.convs[1] = 1;
  a.convs[2] = 0;
  a.filter = 3;
  a.activation = NK_ACT_RELU;
  CHECK(nk_q_size(&a, 32, 32) == 2 * 32 * 32 + 16 * 16);
  CHECK(nk_q_size(&a, 64, 64) == 2 * 64 * 64 + 32 * 32);
  CHECK(nk_q_size(&a, 31, 31) == -1);
  a.convs[0] = 3;
  a.convs[1] = 3;
  a.convs[2] = 3;
  CHECK(nk_q_size(&a, 32, 32) == 3 * (1024 + 256 + 64));
  CHECK(nk_q_size(NULL, 32, 32) == -1);
  if (fails) return 1;
  printf("ok\n");
  return 0;
}
