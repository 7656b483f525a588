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
  // 0: key = (group, crossed-cell bucket).  B > 0: key = (group, spatial
  // block of the ray's start point on a B x B x B grid over the mesh box);
  // the direction is not used (point events of the next-event estimator).
  int32_t blocks_axis;
  // Learned cross sections: when acc_flags is set, rays whose energy lies in
  // [acc_e_lo, acc_e_hi] and in a hash bin with acc_flags[bin] == 0 (the
  // surrogate's accepted bins) take keys below n_groups * n_len, every
  // other ray the same key plus n_groups * n_len (n_keys = 2 n_groups n_len
  // + 1), so the accepted rays come first in the sorted order.
  const uint8_t *acc_flags;
  int32_t acc_n_hash;
  float acc_l2min, acc_inv_bw;
  double acc_e_lo, acc_e_hi;
};

struct RayOut {
  float *x, *y, *z, *u, *v, *w, *E, *wt;
  float4 *aos;  // when set, the sorted rays are written as 32-byte records here
  // optional 32-bit value per ray (input order) carried to the ray's sorted
  // position (single-problem sort only)
  const uint32_t *carry_in;
  uint32_t *carry_out;
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

// ---- batched form: many problems sorted in one pass -------------------------
// Problem p's rays (its own arrays) are sorted by p's key into the
// concatenated output at [ray_base, ray_base + n); the (key, chunk) count
// table holds every problem's block at table_base.
struct BSortProblem {
  SortKeyArgs P;        // key arguments of the problem (chunk field unused)
  const double *edges;  // device group edges or nullptr
  RayPtrs src;          // the problem's rays
  int64_t ray_base;     // first slot in the concatenated output
  int64_t table_base;   // first entry of the problem's (key, chunk) block
  int32_t n_chunks;     // chunks of this problem
  int32_t first_chunk;  // global index of its first chunk
};

struct BSortPlan {
  int chunk = 8192;
  int n_chunks = 0, n_tiles = 0, max_keys = 0;
  int64_t table_len = 0, total_rays = 0;
};

// Launches count / scan / scatter over every problem (5 kernels).
// chunk_problem[c] is the problem of global chunk c.
cudaError_t launch_batched_sort(const BSortProblem *probs_dev, const int32_t *chunk_problem_dev,
                                const BSortPlan &plan, uint32_t *keys, uint32_t *table,
                                uint32_t *offsets, uint32_t *tiles, const RayOut &out,
                                cudaStream_t s);
cudaError_t prepare_batched_sort(const BSortPlan &plan);
int scan_tile_elems();

// out[i] = in[0] + ... + in[i-1] (uint32, n values); tiles is scratch of
// ceil(n / scan_tile_elems()) values.  Three kernel launches on stream s.
cudaError_t launch_exclusive_scan(const uint32_t *in, int64_t n, uint32_t *out, uint32_t *tiles,
                                  cudaStream_t s);

// Makes the single-problem sort kernels resident on the current device
// (cudaFuncGetAttributes on each): under lazy module loading, this is when
// their code is placed on the device.
cudaError_t load_sort_kernels();

// Sort-key arguments, group edges (device), device and stream of a context.
int ctx_sort_args(const vrc_ctx *c, SortKeyArgs *P, const double **edges, int *device,
                  cudaStream_t *stream);

// Records a message for vrc_last_error() and returns code.
int set_last_error(int code, const char *msg);

}  // namespace vrc
