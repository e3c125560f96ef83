/* A plain C caller of the library: builds the surrogate trees of two
 * tetrahedra on the host, then creates a context.  Without a GPU the create
 * call returns MRDEM_ERR_CUDA and the program stops there; with one it runs a
 * detection on device buffers the program allocates itself.  Exit code 0
 * means every status was the expected one. */
#include <stdio.h>
#include <stdint.h>

#include "mrdem.h"

int main(void) {
  /* two unit tetrahedra, the second moved along +x */
  const float verts[2 * 4 * 3] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1,
                                  0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1};
  const int32_t tris[2 * 4 * 3] = {0, 2, 1, 0, 1, 3, 0, 3, 2, 1, 2, 3,
                                   0, 2, 1, 0, 1, 3, 0, 3, 2, 1, 2, 3};
  const int64_t vert_off[3] = {0, 4, 8}, tri_off[3] = {0, 4, 8};
  mrdem_params p;
  mrdem_default_params(&p);
  mrdem_hier* h = NULL;
  int st = mrdem_build_hierarchy_host(&p, 2, vert_off, verts, tri_off, tris, &h);
  if (st != MRDEM_OK) {
    printf("build_hierarchy_host: %s\n", mrdem_status_string(st));
    return 1;
  }
  mrdem_hier_info info;
  if (mrdem_hier_get_info(h, &info) != MRDEM_OK || info.n_particles != 2 || info.n_tri != 8) {
    printf("hier_get_info: unexpected\n");
    return 1;
  }
  printf("trees: %d particles, %lld nodes, depth %d\n", info.n_particles,
         (long long)info.n_nodes, info.max_depth);
  /* bad input is rejected, not aborted on: a triangle index out of range */
  const int32_t bad[12] = {0, 2, 9, 0, 1, 3, 0, 3, 2, 1, 2, 3};
  const int64_t one_v[2] = {0, 4}, one_t[2] = {0, 4};
  mrdem_hier* hb = NULL;
  if (mrdem_build_hierarchy_host(&p, 1, one_v, verts, one_t, bad, &hb) != MRDEM_ERR_INVALID) {
    printf("bad triangle index accepted\n");
    return 1;
  }
  mrdem_ctx* ctx = NULL;
  st = mrdem_create(&ctx, 0, &p);
  if (st == MRDEM_ERR_CUDA) {
    printf("create: %s (no GPU here)\n", mrdem_status_string(st));
    mrdem_hier_destroy(h);
    return 0;
  }
  if (st != MRDEM_OK) {
    printf("create: %s\n", mrdem_status_string(st));
    return 1;
  }
  st = mrdem_hier_upload(ctx, h);
  printf("upload: %s\n", mrdem_status_string(st));
  mrdem_hier_destroy(h);
  mrdem_destroy(ctx);
  return st == MRDEM_OK ? 0 : 1;
}
