// Ray sort before the cast: key layout, scratch plan and launcher
// (implementation in vrc_sort.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vrc_internal.h"

struct vrc_ctx;

namespace vrc {

struct SortKeyArgs {
  float lo[3], hi[3], inv_h[3];  // mesh box and 1/spacing (float32 estimate only)
  int32_t n[3];
  int32_t n_groups;
  int32_t n_len;      // length buckets per group
  int32_t len_width;  // crossed cells per length bucket
  int32_t n_keys;     // n_groups * n_len + 1 (the last key holds rejected rays)
  int32_t chunk;      // rays per block (set by launch_sort)
  int32_t edges_off;  // smem byte offset of the staged group edges (set by launch_sort)
};

struct RayOut {
  float *x, *y, *z, *u, *v, *w, *E, *wt;
};

struct SortPlan {
  int chunk = 0, n_chunks = 0, n_tiles = 0;
  int64_t table_len = 0;
  size_t bytes_keys = 0, bytes_table = 0, bytes_tiles = 0, bytes_rays = 0;
};

SortPlan make_sort_plan(int64_t n, int n_keys);

// Sorts `in` into `out` by key; keys/table/offsets/tiles are scratch of the
// sizes in the plan.  Five kernel launches on stream s.
cudaError_t launch_sort(const RayPtrs &in, SortKeyArgs P, const double *edges, const SortPlan &plan,
                        uint32_t *keys, uint32_t *table, uint32_t *offsets, uint32_t *tiles,
                        const RayOut &out, cudaStream_t s);

// Sort-key arguments, group edges (device), device and stream of a context.
int ctx_sort_args(const vrc_ctx *c, SortKeyArgs *P, const double **edges, int *device,
                  cudaStream_t *stream);

// Records a message for vrc_last_error() and returns code.
int set_last_error(int code, const char *msg);

}  // namespace vrc
