// Ray sort before the cast (no counterpart in the paper, which casts rays in
// buffer order, Sec. 3).  A counting sort on the key
//     key = group * n_len + length bucket   (rejected / out-of-group rays last)
// puts the rays of one energy group together, so that the group's slice of
// the tally stays resident in L2 while it is being scored, and orders each
// group's rays by the number of cells they cross, so that the 32 rays of a
// warp walk about the same number of steps.
//
// Three passes over fixed-size chunks of rays (one chunk per block):
//   k_sort_count   key of every ray; per-chunk histogram written key-major
//   scan           exclusive prefix sum over (key, chunk) -> write offsets
//   k_sort_scatter every ray copied to its slot in the sorted arrays
// Scratch: keys (4 B/ray), the (key, chunk) table, and the sorted rays.
#include <algorithm>

#include "vrc_device.cuh"
#include "vrc_sort.h"

namespace vrc {

namespace {

constexpr int kSortBlock = 256;
constexpr int kSortUnroll = 4;  // rays each sort thread handles at a time

__device__ __forceinline__ int floor_clamp_f(float c, int n) {
  float f = floorf(c);
  f = fminf(fmaxf(f, 0.f), (float)(n - 1));
  return (int)f;
}

// Number of cells the ray crosses, estimated in float32 from its entry and
// exit cells (an ordering key only; the cast does its own exact walk).
__device__ __forceinline__ int crossing_estimate(const SortKeyArgs &P, float px, float py, float pz,
                                                 float u, float v, float w) {
  const float p[3] = {px, py, pz};
  const float d[3] = {u, v, w};
  float s_in = 0.f, s_out = INFINITY;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float lo = P.lo[k], hi = P.hi[k];
    if (d[k] == 0.f) {
      if (p[k] < lo || p[k] >= hi) return 0;
    } else {
      float a = (lo - p[k]) / d[k], b = (hi - p[k]) / d[k];
      if (a > b) { float t = a; a = b; b = t; }
      s_in = fmaxf(s_in, a);
      s_out = fminf(s_out, b);
    }
  }
  if (!(s_in < s_out)) return 0;
  int cells = 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i0 = floor_clamp_f((p[k] + s_in * d[k] - P.lo[k]) * P.inv_h[k], P.n[k]);
    const int i1 = floor_clamp_f((p[k] + s_out * d[k] - P.lo[k]) * P.inv_h[k], P.n[k]);
    cells += abs(i1 - i0);
  }
  return cells;
}

__device__ __forceinline__ uint32_t ray_key(const SortKeyArgs &P, const double *edges, const RayPtrs &R,
                                            int64_t r) {
  float f[8];
  load_ray(R, r, f);
  const float x = f[0], y = f[1], z = f[2], u = f[3], v = f[4], w = f[5], E = f[6], wt = f[7];
  const float dn = norm3(u, v, w);
  const uint32_t reject = (uint32_t)(P.n_keys - 1);
  if (P.blocks_axis > 0) {  // point events: position, energy and weight only
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(E) && isfinite(wt) && E > 0.f)) return reject;
    const int g = group_of(edges, P.n_groups, (double)E);
    if (g < 0) return reject;
    const float p[3] = {x, y, z};
    int b = 0;
#pragma unroll
    for (int k = 2; k >= 0; --k) {
      const float f = (p[k] - P.lo[k]) / (P.hi[k] - P.lo[k]) * (float)P.blocks_axis;
      const int bk = f >= 0.f ? min((int)f, P.blocks_axis - 1) : 0;  // also clamps NaN-free outside starts
      b = b * P.blocks_axis + bk;
    }
    return (uint32_t)(g * P.blocks_axis * P.blocks_axis * P.blocks_axis + b);
  }
  if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(u) && isfinite(v) && isfinite(w) &&
        isfinite(E) && isfinite(wt) && E > 0.f && dn > 0.f && isfinite(dn)))
    return reject;
  const int g = group_of(edges, P.n_groups, (double)E);
  if (g < 0) return reject;
  int c = crossing_estimate(P, x, y, z, u, v, w);
  int b = min(c / P.len_width, P.n_len - 1);
  uint32_t key = (uint32_t)(g * P.n_len + b);
  if (P.acc_flags) {  // rays outside the surrogate's accepted bins go after all accepted ones
    bool acc = false;
    const double e = (double)E;
    if (e >= P.acc_e_lo && e <= P.acc_e_hi) {
      int bin = (int)((__log2f(E) - P.acc_l2min) * P.acc_inv_bw);
      bin = min(max(bin, 0), P.acc_n_hash - 1);
      acc = P.acc_flags[bin] == 0;
    }
    if (!acc) key += (uint32_t)(P.n_groups * P.n_len);
  }
  return key;
}

__global__ void __launch_bounds__(kSortBlock) k_sort_count(RayPtrs R, SortKeyArgs P, const double *edges_g,
                                                           uint32_t *keys, uint32_t *table) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
  double *edges_s = reinterpret_cast<double *>(smem + P.edges_off);
  for (int t = threadIdx.x; t < P.n_keys; t += blockDim.x) hist[t] = 0;
  if (edges_g)
    for (int t = threadIdx.x; t <= P.n_groups; t += blockDim.x) edges_s[t] = edges_g[t];
  __syncthreads();
  const double *edges = edges_g ? edges_s : nullptr;
  const int64_t begin = (int64_t)blockIdx.x * P.chunk;
  const int64_t end = min(begin + P.chunk, R.n);
  for (int64_t r0 = begin + threadIdx.x; r0 < end; r0 += (int64_t)kSortUnroll * blockDim.x) {
    uint32_t k[kSortUnroll];
#pragma unroll
    for (int u = 0; u < kSortUnroll; ++u) {
      const int64_t r = r0 + (int64_t)u * blockDim.x;
      if (r < end) k[u] = ray_key(P, edges, R, r);
    }
#pragma unroll
    for (int u = 0; u < kSortUnroll; ++u) {
      const int64_t r = r0 + (int64_t)u * blockDim.x;
      if (r >= end) break;
      keys[r] = k[u];
      atomicAdd(&hist[k[u]], 1u);
    }
  }
  __syncthreads();
  const int nb = gridDim.x;
  for (int t = threadIdx.x; t < P.n_keys; t += blockDim.x) table[(int64_t)t * nb + blockIdx.x] = hist[t];
}

// Exclusive scan of n uint32 in three kernels: per-tile sums, a scan of the
// tile sums in one block, then per-tile scans with the tile's base.
constexpr int kScanBlock = 1024;
constexpr int kScanTile = 8192;  // elements per tile (8 per thread)

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  uint32_t base = wid > 0 ? warp_sums[wid - 1] : 0u;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  return base + x - v;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(const uint32_t *in, int64_t n, uint32_t *tile_sums) {
  __shared__ uint32_t red[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
  for (int64_t i = base + threadIdx.x; i < min(base + kScanTile, n); i += blockDim.x) s += in[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0u;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(uint32_t *sums, int n) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    uint32_t v = i < n ? sums[i] : 0u;
    uint32_t total;
    uint32_t ex = block_exclusive_scan(v, warp_sums, &total);
    uint32_t c = carry;
    if (i < n) sums[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(const uint32_t *in, int64_t n, const uint32_t *tile_base,
                                                          uint32_t *out) {
  __shared__ uint32_t warp_sums[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  constexpr int per = kScanTile / kScanBlock;
  uint32_t v[per];
  uint32_t local = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    int64_t i = base + (int64_t)threadIdx.x * per + j;
    v[j] = i < n ? in[i] : 0u;
    local += v[j];
  }
  uint32_t ex = block_exclusive_scan(local, warp_sums, nullptr) + tile_base[blockIdx.x];
#pragma unroll
  for (int j = 0; j < per; ++j) {
    int64_t i = base + (int64_t)threadIdx.x * per + j;
    if (i < n) out[i] = ex;
    ex += v[j];
  }
}

__global__ void __launch_bounds__(kSortBlock) k_sort_scatter(RayPtrs R, SortKeyArgs P, const uint32_t *keys,
                                                             const uint32_t *offsets, RayOut O) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *cursor = reinterpret_cast<uint32_t *>(smem);
  const int nb = gridDim.x;
  for (int t = threadIdx.x; t < P.n_keys; t += blockDim.x) cursor[t] = offsets[(int64_t)t * nb + blockIdx.x];
  __syncthreads();
  const int64_t begin = (int64_t)blockIdx.x * P.chunk;
  const int64_t end = min(begin + P.chunk, R.n);
  // kSortUnroll rays per thread at a time: their keys and fields are loaded
  // before any is placed
  for (int64_t r0 = begin + threadIdx.x; r0 < end; r0 += (int64_t)kSortUnroll * blockDim.x) {
    uint32_t key[kSortUnroll];
    float f[kSortUnroll][8];
#pragma unroll
    for (int u = 0; u < kSortUnroll; ++u) {
      const int64_t r = r0 + (int64_t)u * blockDim.x;
      key[u] = r < end ? keys[r] : 0u;
      if (r < end) load_ray(R, r, f[u]);
    }
#pragma unroll
    for (int u = 0; u < kSortUnroll; ++u) {
      const int64_t r = r0 + (int64_t)u * blockDim.x;
      if (r >= end) break;
      const uint32_t pos = atomicAdd(&cursor[key[u]], 1u);
      if (O.aos) {
        O.aos[2 * (int64_t)pos] = make_float4(f[u][0], f[u][1], f[u][2], f[u][3]);
        O.aos[2 * (int64_t)pos + 1] = make_float4(f[u][4], f[u][5], f[u][6], f[u][7]);
      } else {
        O.x[pos] = f[u][0]; O.y[pos] = f[u][1]; O.z[pos] = f[u][2]; O.u[pos] = f[u][3];
        O.v[pos] = f[u][4]; O.w[pos] = f[u][5]; O.E[pos] = f[u][6]; O.wt[pos] = f[u][7];
      }
      if (O.carry_out) O.carry_out[pos] = O.carry_in[r];
    }
  }
}

// ---- batched form -----------------------------------------------------------
__global__ void __launch_bounds__(kSortBlock) k_bsort_count(const BSortProblem *__restrict__ probs,
                                                            const int32_t *__restrict__ chunk_problem,
                                                            int chunk, uint32_t *keys, uint32_t *table) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
  const int p = chunk_problem[blockIdx.x];
  const BSortProblem &B = probs[p];
  const SortKeyArgs P = B.P;
  const int c = blockIdx.x - B.first_chunk;
  for (int t = threadIdx.x; t < P.n_keys; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  const int64_t begin = (int64_t)c * chunk;
  const int64_t end = min(begin + chunk, B.src.n);
  for (int64_t r = begin + threadIdx.x; r < end; r += blockDim.x) {
    uint32_t k = ray_key(P, B.edges, B.src, r);
    keys[B.ray_base + r] = k;
    atomicAdd(&hist[k], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P.n_keys; t += blockDim.x)
    table[B.table_base + (int64_t)t * B.n_chunks + c] = hist[t];
}

__global__ void __launch_bounds__(kSortBlock) k_bsort_scatter(const BSortProblem *__restrict__ probs,
                                                              const int32_t *__restrict__ chunk_problem,
                                                              int chunk, const uint32_t *keys,
                                                              const uint32_t *offsets, RayOut O) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *cursor = reinterpret_cast<uint32_t *>(smem);
  const int p = chunk_problem[blockIdx.x];
  const BSortProblem &B = probs[p];
  const int n_keys = B.P.n_keys;
  const int c = blockIdx.x - B.first_chunk;
  for (int t = threadIdx.x; t < n_keys; t += blockDim.x)
    cursor[t] = offsets[B.table_base + (int64_t)t * B.n_chunks + c];
  __syncthreads();
  const int64_t begin = (int64_t)c * chunk;
  const int64_t end = min(begin + chunk, B.src.n);
  const RayPtrs R = B.src;
  for (int64_t r = begin + threadIdx.x; r < end; r += blockDim.x) {
    const uint32_t pos = atomicAdd(&cursor[keys[B.ray_base + r]], 1u);
    float f[8];
    load_ray(R, r, f);
    if (O.aos) {
      O.aos[2 * (int64_t)pos] = make_float4(f[0], f[1], f[2], f[3]);
      O.aos[2 * (int64_t)pos + 1] = make_float4(f[4], f[5], f[6], f[7]);
    } else {
      O.x[pos] = f[0]; O.y[pos] = f[1]; O.z[pos] = f[2]; O.u[pos] = f[3];
      O.v[pos] = f[4]; O.w[pos] = f[5]; O.E[pos] = f[6]; O.wt[pos] = f[7];
    }
  }
}

size_t count_smem(const SortKeyArgs &P) {
  return (size_t)P.edges_off + sizeof(double) * (size_t)(P.n_groups + 1);
}

}  // namespace

SortPlan make_sort_plan(int64_t n, int n_keys) {
  SortPlan p;
  p.chunk = 8192;
  p.n_chunks = (int)((n + p.chunk - 1) / p.chunk);
  p.table_len = (int64_t)n_keys * p.n_chunks;
  p.n_tiles = (int)((p.table_len + kScanTile - 1) / kScanTile);
  p.bytes_keys = sizeof(uint32_t) * (size_t)n;
  p.bytes_table = sizeof(uint32_t) * (size_t)p.table_len;
  p.bytes_tiles = sizeof(uint32_t) * (size_t)p.n_tiles;
  p.bytes_rays = 8 * sizeof(float) * (size_t)n;
  return p;
}

cudaError_t launch_sort(const RayPtrs &in, SortKeyArgs P, const double *edges, const SortPlan &plan,
                        uint32_t *keys, uint32_t *table, uint32_t *offsets, uint32_t *tiles,
                        const RayOut &out, cudaStream_t s) {
  if (in.n == 0) return cudaSuccess;
  P.chunk = plan.chunk;
  P.edges_off = (int)(((size_t)P.n_keys * sizeof(uint32_t) + 15) / 16 * 16);
  const size_t smem_count = count_smem(P);
  const size_t smem_scatter = sizeof(uint32_t) * (size_t)P.n_keys;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_sort_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_count)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_scatter)) != cudaSuccess) return e;
  k_sort_count<<<plan.n_chunks, kSortBlock, smem_count, s>>>(in, P, edges, keys, table);
  k_scan_tiles<<<plan.n_tiles, kScanBlock, 0, s>>>(table, plan.table_len, tiles);
  k_scan_sums<<<1, kScanBlock, 0, s>>>(tiles, plan.n_tiles);
  k_scan_apply<<<plan.n_tiles, kScanBlock, 0, s>>>(table, plan.table_len, tiles, offsets);
  k_sort_scatter<<<plan.n_chunks, kSortBlock, smem_scatter, s>>>(in, P, keys, offsets, out);
  note_launches(5);
  return cudaGetLastError();
}

cudaError_t prepare_batched_sort(const BSortPlan &plan) {
  const int smem = (int)(sizeof(uint32_t) * (size_t)plan.max_keys);
  cudaError_t e = cudaFuncSetAttribute(k_bsort_count, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_bsort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_batched_sort(const BSortProblem *probs_dev, const int32_t *chunk_problem_dev,
                                const BSortPlan &plan, uint32_t *keys, uint32_t *table,
                                uint32_t *offsets, uint32_t *tiles, const RayOut &out,
                                cudaStream_t s) {
  if (plan.n_chunks == 0) return cudaSuccess;
  const size_t smem = sizeof(uint32_t) * (size_t)plan.max_keys;
  k_bsort_count<<<plan.n_chunks, kSortBlock, smem, s>>>(probs_dev, chunk_problem_dev, plan.chunk, keys, table);
  k_scan_tiles<<<plan.n_tiles, kScanBlock, 0, s>>>(table, plan.table_len, tiles);
  k_scan_sums<<<1, kScanBlock, 0, s>>>(tiles, plan.n_tiles);
  k_scan_apply<<<plan.n_tiles, kScanBlock, 0, s>>>(table, plan.table_len, tiles, offsets);
  k_bsort_scatter<<<plan.n_chunks, kSortBlock, smem, s>>>(probs_dev, chunk_problem_dev, plan.chunk, keys, offsets, out);
  note_launches(5);
  return cudaGetLastError();
}

int scan_tile_elems() { return kScanTile; }

cudaError_t launch_exclusive_scan(const uint32_t *in, int64_t n, uint32_t *out, uint32_t *tiles,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int n_tiles = (int)((n + kScanTile - 1) / kScanTile);
  k_scan_tiles<<<n_tiles, kScanBlock, 0, s>>>(in, n, tiles);
  k_scan_sums<<<1, kScanBlock, 0, s>>>(tiles, n_tiles);
  k_scan_apply<<<n_tiles, kScanBlock, 0, s>>>(in, n, tiles, out);
  note_launches(3);
  return cudaGetLastError();
}

cudaError_t load_sort_kernels() {
  cudaFuncAttributes fa;
  const void *fns[] = {(const void *)k_sort_count, (const void *)k_scan_tiles, (const void *)k_scan_sums,
                       (const void *)k_scan_apply, (const void *)k_sort_scatter};
  for (const void *f : fns) {
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace vrc
