// Internal declarations shared by the libvrc translation units (host and
// device).  Not part of the public ABI; see include/vrc.h for that.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vrc {

constexpr int kMaxMaterials = 64;  // material ids are uint8; per-thread sigma lives in smem
constexpr int kMaxGroups = 1024;

// Status bits written by kernels (read by vrc_sync / vrc_read_tally).
constexpr unsigned kStatusNonfinite = 1u;
constexpr unsigned kStatusTraversal = 2u;
constexpr unsigned kStatusTableFull = 4u;  // a per-history table insert found no free slot
constexpr unsigned kStatusTimeout = 8u;    // a bounded wait on the tensor cores gave up

// Device counters (unsigned long long each).
// kCntLive: segments whose score was added to the tally (non-zero; once a
// ray's transmitted fraction is exactly 0 its segments are walked, not scored).
enum Counter { kCntSegments = 0, kCntRays = 1, kCntRejected = 2, kCntOverflow = 3, kCntLive = 4, kNumCounters = 5 };

// A value held as an unevaluated sum hi + lo of two float32 ("double-float").
struct df {
  float hi, lo;
};

// Cartesian mesh, geometry split into double-float pairs on the host.  A
// uniform mesh has planes at org + j h; a rectilinear one (rect != 0) at
// edge[k][j], j = 0..n[k], each plane position as a (hi, lo) float pair.
struct MeshDev {
  int32_t n[3];
  int64_t ncells;
  int64_t stride[3];  // 1, nx, nx*ny
  df org[3];          // x0, y0, z0
  df h[3];            // dx, dy, dz
  df inv_h[3];        // 1/dx, 1/dy, 1/dz
  const uint8_t *mat; // [nz][ny][nx]
  const float2 *edge[3];
  int32_t rect;
};

// Cross sections on the union energy grid of all materials.
struct XsDev {
  int32_t n_union;   // points on the union grid (0 = every material void)
  int32_t m_pad;     // row stride (floats) of S
  int32_t n_mat;     // materials
  int32_t n_hash;    // hash bins over log2(E)
  float l2min;       // log2 of the first grid energy
  float inv_bw;      // bins per unit of log2(E)
  const double *E;      // [n_union] union grid energies (eV)
  const double *inv_dE; // [n_union-1] 1/(E[i+1]-E[i])
  const float *S;       // [n_union][m_pad] sigma_t at the union points
  const int32_t *hash;  // [n_hash+1] interval index at each bin's lower energy
};

// A ray batch: eight float32 arrays (SoA), or, when aos is set, one array
// of 32-byte records (x, y, z, u | v, w, E, wt) as two float4 per ray.
struct RayPtrs {
  const float *x, *y, *z, *u, *v, *w, *E, *wt;
  const float4 *aos;
  int64_t n;
};

// Output of a per-history cast: ray r writes its scores, in walk order, to
// pairs[off[r]] .. pairs[off[r] + cap[r] - 1] as (key, float64 bits), key =
// bin << 32 | history id, bin = group * ncells + cell, and the number
// written to cnt[r] (cap[r] is an upper bound of the ray's segments).  With
// stride != 0, off[r] = r * stride and cap[r] = stride (off, cap unused).
// The cast also counts the pairs it writes per bucket of 2^bshift
// consecutive bins into bcount (zeroed before the cast), one reduction per
// run of a ray's pairs in one bucket.
struct PairOut {
  ulonglong2 *pairs;
  const uint32_t *off;
  const uint32_t *cap;
  uint32_t *cnt;
  uint32_t stride;
  uint32_t *bcount;
  int32_t bshift;
};

__host__ __device__ __forceinline__ uint32_t pair_off(const PairOut &p, int64_t r) {
#ifdef __CUDA_ARCH__
  return p.stride ? (uint32_t)r * p.stride : __ldg(p.off + r);
#else
  return p.stride ? (uint32_t)r * p.stride : p.off[r];
#endif
}
__host__ __device__ __forceinline__ uint32_t pair_cap(const PairOut &p, int64_t r) {
#ifdef __CUDA_ARCH__
  return p.stride ? p.stride : __ldg(p.cap + r);
#else
  return p.stride ? p.stride : p.cap[r];
#endif
}

struct CastArgs {
  MeshDev mesh;
  XsDev xs;
  const double *edges;  // [n_groups+1] or nullptr (single group, every energy)
  int32_t n_groups;
  RayPtrs rays;
  const float *sig_ray; // [n][16] per-ray sigma from the surrogate for rays r < *n_surr, or nullptr
  const uint32_t *n_surr; // device count of leading rays with surrogate sigma (with sig_ray)
  double *tally;        // [n_groups][ncells]
  const uint32_t *hist; // [n] history id of each ray (per-history cast only)
  PairOut pout;         // per-history cast only
  int32_t stop_zero;    // end a walk once its transmitted fraction is exactly 0
  // Ray assignment: 0, each thread takes rays r, r + (grid threads), ...;
  // R > 0 (a multiple of 32), each warp takes R consecutive rays at a time
  // from the counter *queue (zeroed before the launch).
  int32_t rays_per_warp;
  unsigned long long *queue;
  unsigned long long *counters;
  unsigned int *status;
};

// Batched form (vrc_batched.cu): a work item is a chunk of one problem's rays.
struct BatchItem {
  int32_t problem;
  int32_t count;
  int64_t start;
};

// Largest per-problem table sizes in a batch (shared memory is sized by them).
struct BatchShape {
  int32_t max_hash, max_groups, max_mat;
};

size_t batched_smem_bytes(int form, const BatchShape &sh, int block);
cudaError_t batched_occupancy(int form, const BatchShape &sh, int block, int *blocks_per_sm);
// rays_per_warp 0: a block's warps take an item's rays interleaved; R > 0:
// R at a time from the item's counter in shared memory.
cudaError_t launch_batched_cast(int form, const CastArgs *probs, const BatchItem *items, int n_items,
                                unsigned int *queue, const BatchShape &sh, int grid, int block,
                                int rays_per_warp, cudaStream_t s);

// Next-event estimator (vrc_detect.cu): adds every ray's flux at n_det
// detector points (float [n_det][3]) to out [n_det][n_groups] (device).
cudaError_t launch_detectors(int form, const CastArgs &a, const float *det, int n_det, double *out,
                             int num_sms, cudaStream_t s);

// Process-wide count of kernels launched by libvrc (vrc_launch_count).
void note_launches(int n);

// Launchers (vrc_cast.cu).  smem_bytes() gives the dynamic shared memory a
// cast launch of the given block size needs.
size_t cast_smem_bytes(int form, const CastArgs &a, int block);
cudaError_t launch_cast(int form, const CastArgs &a, int grid, int block, cudaStream_t s);
cudaError_t cast_occupancy(int form, const CastArgs &a, int block, int *blocks_per_sm);
cudaError_t launch_scale_copy(const double *src, double *dst, int64_t n, double scale,
                              cudaStream_t s);
// Per-volume copy of a rectilinear tally slice: dst[i] = src[i] / volume of
// cell (first + i) mod ncells, volumes from per-axis widths w[k] (device).
cudaError_t launch_per_volume_rect(const double *src, double *dst, int64_t n, int64_t first, int32_t nx,
                                   int32_t ny, int64_t ncells, const double *wx, const double *wy,
                                   const double *wz, cudaStream_t s);
// Tally moments (vrc_history.cu): mom[bin] = (S1, S2), the sums of the
// samples and of their squares per (group, cell).  Batch moments: the fold
// mom += (t, t^2), t = 0.  Per-history moments: each ray's room in the pair
// buffer (a fixed stretch, or an upper bound of its segments, cap), the cast
// that writes each ray's (key, score) pairs and counts them per bucket of
// 2^shift consecutive bins (vrc_cast.cu), the scatter of the pairs into
// their buckets, and per bucket the sum x of every (history, bin) and
// mom[bin] += (x, x^2).
cudaError_t launch_fold_moments(double *tally, double2 *mom, int64_t n, cudaStream_t s);
struct BoundGeom {
  double lo[3], h[3];
  int32_t n[3];
  const double *e[3];  // rectilinear plane positions (device), or nullptr
};
cudaError_t launch_ray_caps(const BoundGeom &g, const RayPtrs &rays, uint32_t *cap, int num_sms,
                            cudaStream_t s);
cudaError_t launch_cast_hist(int form, const CastArgs &a, int grid, int block, cudaStream_t s);
cudaError_t cast_hist_occupancy(int form, const CastArgs &a, int block, int *blocks_per_sm);
// Bucket sort and fold of the pairs of n_rays rays (PairOut with pairs,
// off or stride, cnt, and bcount / bshift counted by the cast) into mom:
// p.bcount and base hold n_buckets + 1 values (bcount[n_buckets] = 0); tiles
// is scan scratch; sorted receives the pairs bucket by bucket; status gets
// kStatusTableFull if a bucket's shared-memory table overflows.
constexpr int kPairMaxBuckets = 262144;  // buckets of the pair sort, at most
cudaError_t launch_pair_fold(const PairOut &p, int64_t n_rays, int n_buckets, uint32_t *base, uint32_t *tiles,
                             ulonglong2 *sorted, double2 *mom, unsigned int *status, int num_sms,
                             cudaStream_t s);
// total[i] = S1; sigma[i] = sqrt(B/(B-1) (S2 - S1^2/B)) if sigma is not null.
cudaError_t launch_moment_read(const double2 *mom, double *total, double *sigma, int64_t n, double B,
                               cudaStream_t s);

}  // namespace vrc
