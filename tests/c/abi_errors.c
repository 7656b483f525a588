/* C test driver for the libvrc boundary: argument validation and error
 * codes that need no GPU (every case below is rejected before any device
 * work).  Exit status 0 on success; prints the first failing check. */
#include <stdio.h>
#include <string.h>
#include <math.h>
#include "vrc.h"

static int failures = 0;
#define EXPECT(cond)                                                         \
  do {                                                                       \
    if (!(cond)) {                                                           \
      fprintf(stderr, "FAIL %s:%d: %s (last error: %s)\n", __FILE__, __LINE__, \
              #cond, vrc_last_error());                                      \
      ++failures;                                                            \
    }                                                                        \
  } while (0)

int main(void) {
  vrc_options o;
  vrc_default_options(&o);
  EXPECT(o.form == VRC_FORM_PLAIN && o.sort == -1 && o.block == 0 && o.device == -1 && o.stop_at_zero == 0);
  vrc_default_options(NULL); /* must not crash */

  uint8_t mat[8] = {0, 1, 0, 1, 0, 1, 0, 1};
  double edges[3] = {1.0, 10.0, 100.0};
  vrc_mesh_desc d = {2, 2, 2, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, mat, 2, 1, NULL};
  vrc_ctx *c = (vrc_ctx *)0x1;

  EXPECT(vrc_create_mesh(NULL, NULL, &c) == VRC_ERR_ARG && c == NULL);
  EXPECT(vrc_create_mesh(&d, NULL, NULL) == VRC_ERR_ARG);
  vrc_mesh_desc b = d; b.nx = 0;
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  b = d; b.dy = -1.0;
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  b = d; b.dz = NAN;
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  b = d; b.x0 = INFINITY;
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  b = d; b.material = NULL;
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  b = d; b.n_materials = 1; /* material id 1 is out of range */
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  EXPECT(strstr(vrc_last_error(), "material") != NULL);
  b = d; b.n_materials = 65;
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  b = d; b.n_groups = 2; /* edges missing */
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  b = d; b.n_groups = 2; b.group_edges = edges; edges[1] = 0.5; /* not ascending */
  EXPECT(vrc_create_mesh(&b, NULL, &c) == VRC_ERR_ARG);
  edges[1] = 10.0;
  vrc_options bad = o; bad.form = 7;
  EXPECT(vrc_create_mesh(&d, &bad, &c) == VRC_ERR_ARG);
  bad = o; bad.block = 100;
  EXPECT(vrc_create_mesh(&d, &bad, &c) == VRC_ERR_ARG);
  bad = o; bad.block = 512;
  EXPECT(vrc_create_mesh(&d, &bad, &c) == VRC_ERR_ARG);
  bad = o; bad.sort = 2;
  EXPECT(vrc_create_mesh(&d, &bad, &c) == VRC_ERR_ARG);
  bad = o; bad.sort_len_buckets = 0;
  EXPECT(vrc_create_mesh(&d, &bad, &c) == VRC_ERR_ARG);
  bad = o; bad.sort_len_buckets = 300;
  EXPECT(vrc_create_mesh(&d, &bad, &c) == VRC_ERR_ARG);
  bad = o; bad.stop_at_zero = 2;
  EXPECT(vrc_create_mesh(&d, &bad, &c) == VRC_ERR_ARG);

  /* calls on a NULL context */
  double E[2] = {1.0, 2.0}, S[2] = {1.0, 1.0};
  EXPECT(vrc_load_xs(NULL, 0, E, S, 2) == VRC_ERR_ARG);
  vrc_rays r;
  memset(&r, 0, sizeof r);
  EXPECT(vrc_cast_rays(NULL, &r, NULL) == VRC_ERR_ARG);
  EXPECT(vrc_sync(NULL, NULL, NULL) == VRC_ERR_ARG);
  double out[8];
  EXPECT(vrc_read_tally(NULL, out, 8, 0, NULL) == VRC_ERR_ARG);
  EXPECT(vrc_reset_tally(NULL, NULL) == VRC_ERR_ARG);
  EXPECT(vrc_set_options(NULL, &o) == VRC_ERR_ARG);
  EXPECT(vrc_tally_device_ptr(NULL) == NULL);
  vrc_destroy(NULL); /* no-op */

  /* batched form */
  vrc_batch_options bo;
  vrc_default_batch_options(&bo);
  EXPECT(bo.use_graph == 1 && bo.sort_len_buckets == -1 && bo.chunk == 0);
  vrc_batch *bt = (vrc_batch *)0x1;
  EXPECT(vrc_batch_create(NULL, &r, 1, NULL, &bt) == VRC_ERR_ARG && bt == NULL);
  vrc_ctx *none[1] = {NULL};
  EXPECT(vrc_batch_create(none, &r, 1, NULL, &bt) == VRC_ERR_ARG);
  EXPECT(vrc_batch_create(none, &r, 0, NULL, &bt) == VRC_ERR_ARG);
  vrc_batch_options bb = bo; bb.chunk = 10;
  EXPECT(vrc_batch_create(none, &r, 1, &bb, &bt) == VRC_ERR_ARG);
  bb = bo; bb.block = 48;
  EXPECT(vrc_batch_create(none, &r, 1, &bb, &bt) == VRC_ERR_ARG);
  bb = bo; bb.rays_per_warp = 48;
  EXPECT(vrc_batch_create(none, &r, 1, &bb, &bt) == VRC_ERR_ARG);
  EXPECT(vrc_batch_launch(NULL, NULL) == VRC_ERR_ARG);
  vrc_batch_destroy(NULL);
  EXPECT(vrc_cast_batched(NULL, &r, 1, NULL) == VRC_ERR_ARG);
  EXPECT(vrc_sort_rays_static(NULL, &r, NULL, NULL) == VRC_ERR_ARG);

  /* rectilinear meshes: edge checks come before any device work */
  double xe[3] = {0.0, 0.5, 2.0}, ye[3] = {-1.0, 0.0, 1.0}, ze[3] = {0.0, 3.0, 4.0};
  vrc_rect_mesh_desc rd = {2, 2, 2, xe, ye, ze, mat, 2, 1, NULL};
  EXPECT(vrc_create_rect_mesh(NULL, NULL, &c) == VRC_ERR_ARG && c == NULL);
  EXPECT(vrc_create_rect_mesh(&rd, NULL, NULL) == VRC_ERR_ARG);
  vrc_rect_mesh_desc rb = rd; rb.y_edges = NULL;
  EXPECT(vrc_create_rect_mesh(&rb, NULL, &c) == VRC_ERR_ARG);
  xe[1] = 0.0; /* not strictly ascending */
  EXPECT(vrc_create_rect_mesh(&rd, NULL, &c) == VRC_ERR_ARG);
  EXPECT(strstr(vrc_last_error(), "ascending") != NULL);
  xe[1] = NAN;
  EXPECT(vrc_create_rect_mesh(&rd, NULL, &c) == VRC_ERR_ARG);
  xe[1] = 0.5;
  rb = rd; rb.nz = 0;
  EXPECT(vrc_create_rect_mesh(&rb, NULL, &c) == VRC_ERR_ARG);

  /* moments and per-history casts on a NULL context */
  uint32_t hist[1] = {0};
  EXPECT(vrc_moments_enable(NULL, VRC_MOMENTS_HISTORY) == VRC_ERR_ARG);
  EXPECT(vrc_moments_fold(NULL, NULL) == VRC_ERR_ARG);
  EXPECT(vrc_cast_histories(NULL, &r, hist, 1, NULL) == VRC_ERR_ARG);
  EXPECT(vrc_context_stream(NULL) == NULL);
  /* the allocation-failure hook touches no GPU */
  EXPECT(vrc_debug_fail_alloc(3) == VRC_OK);
  EXPECT(vrc_debug_fail_alloc(-1) == VRC_OK);
  EXPECT(vrc_version() == VRC_VERSION);
  EXPECT(vrc_device_count() >= 0);

  if (failures) return 1;
  printf("abi_errors: all checks passed\n");
  return 0;
}
