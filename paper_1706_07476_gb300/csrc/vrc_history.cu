// Tally moments (the sums behind the tally's standard deviation in Eqs. 5
// and 8), kept as (S1, S2) pairs per (group, cell): the batch fold, the read
// (S1 and sigma), and for per-history moments the room of each ray in the
// pair buffer and the fold of a per-history cast's (key, score) pairs into
// S1 += x, S2 += x^2, x the summed score of one history in one bin.
#include <algorithm>
#include <math.h>

#include "vrc_internal.h"
#include "vrc_sort.h"

namespace vrc {

namespace {

__device__ __forceinline__ double plane_lo(const BoundGeom &G, int k) {
  return G.e[k] ? G.e[k][0] : G.lo[k];
}
__device__ __forceinline__ double plane_hi(const BoundGeom &G, int k) {
  return G.e[k] ? G.e[k][G.n[k]] : G.lo[k] + G.h[k] * G.n[k];
}

// Cell index on axis k of coordinate q, clamped (uniform: floor; rectilinear:
// binary search on the plane positions).
__device__ __forceinline__ double cell_of(const BoundGeom &G, int k, double q) {
  const int n = G.n[k];
  if (!G.e[k]) return fmin(fmax(floor((q - G.lo[k]) / G.h[k]), 0.0), n - 1.0);
  const double *e = G.e[k];
  if (!(q >= e[0])) return 0.0;
  if (q >= e[n]) return n - 1.0;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (e[mid] <= q) lo = mid; else hi = mid;
  }
  return (double)lo;
}

// Upper bound of the cells one ray crosses: the ray p + s d is clipped to
// the box in float64, and the cell indices at its entry and exit differ by
// the planes it crosses on each axis; one cell more, plus one per axis for
// rounding differences from the walk.  Rays that miss the box, or that the
// cast rejects (non-finite, zero direction), count 0.
__device__ __forceinline__ unsigned long long ray_bound(const BoundGeom &G, const float f[6]) {
  const double p[3] = {f[0], f[1], f[2]};
  const double d[3] = {f[3], f[4], f[5]};
  if (!(d[0] != 0.0 || d[1] != 0.0 || d[2] != 0.0)) return 0;
  double s_in = 0.0, s_out = INFINITY;
  for (int k = 0; k < 3; ++k) {
    const double lo = plane_lo(G, k), hi = plane_hi(G, k);
    if (d[k] == 0.0) {
      if (!(p[k] >= lo && p[k] < hi)) return 0;
    } else {
      double a = (lo - p[k]) / d[k], b = (hi - p[k]) / d[k];
      if (d[k] < 0.0) { const double t = a; a = b; b = t; }
      s_in = fmax(s_in, a);
      s_out = fmin(s_out, b);
    }
  }
  if (!(s_in < s_out)) return 0;  // also false for NaN
  unsigned long long cells = 1 + 3;
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0) continue;
    const double a = cell_of(G, k, p[k] + s_in * d[k]);
    const double b = cell_of(G, k, p[k] + s_out * d[k]);
    cells += (unsigned long long)fabs(b - a);
  }
  return cells;
}

// ray_bound on a uniform mesh in float32 arithmetic: the clipped entry and
// exit points can each be one cell off per axis in float32, so the margin is
// two cells per axis more than ray_bound's.
__device__ __forceinline__ unsigned long long ray_bound_f(const BoundGeom &G, const float f[6]) {
  if (!(f[3] != 0.f || f[4] != 0.f || f[5] != 0.f)) return 0;
  float s_in = 0.f, s_out = INFINITY;
  for (int k = 0; k < 3; ++k) {
    const float lo = (float)G.lo[k], hi = (float)(G.lo[k] + G.h[k] * G.n[k]);
    if (f[3 + k] == 0.f) {
      if (!(f[k] >= lo && f[k] < hi)) return 0;
    } else {
      const float inv = 1.f / f[3 + k];
      float a = (lo - f[k]) * inv, b = (hi - f[k]) * inv;
      if (inv < 0.f) { const float t = a; a = b; b = t; }
      s_in = fmaxf(s_in, a);
      s_out = fminf(s_out, b);
    }
  }
  if (!(s_in < s_out)) return 1 + 3 + 6;  // a near miss: the walk may still clip a corner
  unsigned long long cells = 1 + 3 + 6;
  for (int k = 0; k < 3; ++k) {
    if (f[3 + k] == 0.f) continue;
    const float ih = (float)(1.0 / G.h[k]), lo = (float)G.lo[k], nm1 = (float)(G.n[k] - 1);
    const float a = fminf(fmaxf(floorf((fmaf(s_in, f[3 + k], f[k]) - lo) * ih), 0.f), nm1);
    const float b = fminf(fmaxf(floorf((fmaf(s_out, f[3 + k], f[k]) - lo) * ih), 0.f), nm1);
    cells += (unsigned long long)fabsf(b - a);
  }
  return cells;
}

// Room of every ray in the pair buffer: an upper bound of its segments
// (float32 on a uniform mesh, float64 on a rectilinear one), capped at
// 2^32 - 1.
__global__ void k_ray_caps(BoundGeom G, RayPtrs R, uint32_t *cap) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R.n;
       r += (int64_t)gridDim.x * blockDim.x) {
    float f[6];
    if (R.aos) {
      const float4 a = R.aos[2 * r], b = R.aos[2 * r + 1];
      f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y;
    } else {
      f[0] = R.x[r]; f[1] = R.y[r]; f[2] = R.z[r]; f[3] = R.u[r]; f[4] = R.v[r]; f[5] = R.w[r];
    }
    const bool ok = isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]) && isfinite(f[3]) && isfinite(f[4]) &&
                    isfinite(f[5]);
    const unsigned long long b = !ok ? 0ull : (G.e[0] ? ray_bound(G, f) : ray_bound_f(G, f));
    cap[r] = b < 0xffffffffull ? (uint32_t)b : 0xffffffffu;
  }
}

// ---- fold of the per-history pairs ------------------------------------------
// A counting sort puts the pairs into buckets of 2^shift consecutive bins
// (the cast counts each bucket's pairs; a scan gives the buckets' first
// slots; k_pair_scatter moves the pairs); then one block per bucket sums
// the scores of equal keys (history, bin) in a shared-memory hash table and
// adds (x, x^2) to the bin's moments.  A bucket's bins are a contiguous stretch of the moment
// array, so those reductions stay in L2.  A bucket with more keys than 0.7
// of the table is folded in several passes, each over the keys whose hash
// falls in that pass.
constexpr int kFoldThreads = 256;  // threads per block of the scatter
// The fold's shared-memory hash table (16 bytes a slot), threads and blocks
// per SM.  Small blocks, many per SM, each on a small bucket (kPairMaxBuckets
// of them: about 150 keys each for 2^20 slab256 rays, filling 60 % of a
// table) measured fastest: a block waits at its barriers for 2 warps only.
constexpr int kFoldSlots = 256;
constexpr int kFoldBlockThreads = 64;
constexpr int kFoldBlocksPerSm = 32;
constexpr int kFoldPassKeys = kFoldSlots * 7 / 10;  // keys per pass: load factor at most 0.7
constexpr unsigned long long kEmptyKey = ~0ull;  // bin 2^32 - 1 never occurs

// Scatter of the pairs into buckets: each pair goes to cursor[b]++, where
// cursor[b] starts at bucket b's first slot (the scan of the counts the cast
// took).  Each warp takes 32 consecutive rays at a time (a grid-stride loop
// over groups of 32) and spreads their pairs over its lanes: lane l handles
// pairs j + l of the group's pairs in a row (the ray of a pair found by a
// binary search over the warp's prefix sums of the counts), so consecutive
// lanes read consecutive pairs; four such rounds are loaded before any is
// used.  A run of consecutive lanes with the same bucket (mostly
// consecutive pairs of one ray) shares one global atomic, taken by the
// run's first lane (a lane whose bucket differs from the lane before it).
__global__ void __launch_bounds__(kFoldThreads) k_pair_scatter(PairOut P, int64_t n_rays, uint32_t *cursor,
                                                               ulonglong2 *sorted) {
  const unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int shift = P.bshift;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < n_rays;
       r0 += 32 * warps) {
    const int64_t r = r0 + lane;
    const uint32_t n = r < n_rays ? P.cnt[r] : 0u;
    const uint32_t o = r < n_rays ? pair_off(P, r) : 0u;
    uint32_t incl = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(kAll, incl, d);
      if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(kAll, incl, 31), excl = incl - n;
    for (uint32_t base = 0; base < total; base += 4 * 32) {
      ulonglong2 q[4];
      bool valid[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t t = base + 32 * u + lane;
        int k = 0;  // the last ray whose pairs start at or before t
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t e = __shfl_sync(kAll, excl, k + step);
          if (e <= t) k += step;
        }
        const uint32_t ok = __shfl_sync(kAll, o, k), ek = __shfl_sync(kAll, excl, k);
        valid[u] = t < total;
        q[u] = valid[u] ? P.pairs[ok + (t - ek)] : make_ulonglong2(0ull, 0ull);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t b = valid[u] ? (uint32_t)(q[u].x >> 32) >> shift : 0xffffffffu;
        const uint32_t prev = __shfl_up_sync(kAll, b, 1);
        const unsigned heads = __ballot_sync(kAll, lane == 0 || b != prev);
        // this lane's run: from its head (the last head at or below it) to
        // the lane before the next head
        const int head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const unsigned above = heads & ~(0xffffffffu >> (31 - lane));
        const int next = above ? __ffs(above) - 1 : 32;
        uint32_t first = 0;
        if (valid[u] && lane == head) first = atomicAdd(cursor + b, (uint32_t)(next - head));
        first = __shfl_sync(kAll, first, head);
        if (valid[u]) sorted[first + (uint32_t)(lane - head)] = q[u];
      }
    }
  }
}

// 32-bit hash of a pair key (history in the low word, bin in the high one).
__device__ __forceinline__ uint32_t key_hash(unsigned long long k) {
  uint32_t h = (uint32_t)k * 0x9E3779B1u ^ (uint32_t)(k >> 32) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  return h ^ (h >> 13);
}

__global__ void __launch_bounds__(kFoldBlockThreads, kFoldBlocksPerSm) k_pair_fold(const ulonglong2 *__restrict__ sorted,
                                                                    const uint32_t *__restrict__ base,
                                                                    int n_buckets, double2 *__restrict__ mom,
                                                                    unsigned int *status) {
  extern __shared__ unsigned long long keys[];  // [kFoldSlots], then the sums [kFoldSlots]
  double *vals = reinterpret_cast<double *>(keys + kFoldSlots);
  // the table starts empty; every drain leaves the slots it used empty again
  for (int t = threadIdx.x; t < kFoldSlots; t += blockDim.x) { keys[t] = kEmptyKey; vals[t] = 0.0; }
  __syncthreads();
  for (int b = blockIdx.x; b < n_buckets; b += gridDim.x) {
    const uint32_t begin = base[b], end = base[b + 1];
    if (begin == end) continue;
    // a table sized to the bucket, or several passes of the full table, each
    // over the keys whose hash falls in it
    const uint32_t count = end - begin;
    const uint32_t passes = (count + kFoldPassKeys - 1) / kFoldPassKeys;
    uint32_t slots = 64, lg = 6;
    while (10 * count > 7 * slots && slots < (uint32_t)kFoldSlots) { slots <<= 1; ++lg; }
    for (uint32_t p = 0; p < passes; ++p) {
      bool full = false;
      for (uint32_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        const ulonglong2 q = sorted[i];
        const uint32_t h = key_hash(q.x);
        if (passes > 1 && h % passes != p) continue;
        uint32_t slot = h >> (32 - lg);
        uint32_t probe = 0;
        for (; probe < slots; ++probe) {
          const unsigned long long old = atomicCAS(&keys[slot], kEmptyKey, q.x);
          if (old == kEmptyKey || old == q.x) break;
          slot = (slot + 1) & (slots - 1);
        }
        if (probe == slots) { full = true; continue; }
        atomicAdd(&vals[slot], __longlong_as_double((long long)q.y));
      }
      if (full) atomicOr(status, kStatusTableFull);
      __syncthreads();
      for (uint32_t t = threadIdx.x; t < slots; t += blockDim.x) {
        const unsigned long long k = keys[t];
        if (k == kEmptyKey) continue;
        const double x = vals[t];
        keys[t] = kEmptyKey;
        vals[t] = 0.0;
        double2 *m = mom + (k >> 32);
        atomicAdd(&m->x, x);
        atomicAdd(&m->y, x * x);
      }
      __syncthreads();
    }
  }
}

// Batch moments: mom += (t, t^2), t = 0.
__global__ void k_fold_moments(double *__restrict__ t, double2 *__restrict__ mom, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = t[i];
    const double2 m = mom[i];
    mom[i] = make_double2(m.x + v, fma(v, v, m.y));
    t[i] = 0.0;
  }
}

// total = S1; sigma = sqrt(B/(B-1) (S2 - S1^2/B)), clamped at 0 against
// rounding (Eqs. 5 and 8 take the standard deviation of the tally).
__global__ void k_moment_read(const double2 *__restrict__ mom, double *__restrict__ total,
                              double *__restrict__ sigma, int64_t n, double B) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 m = mom[i];
    total[i] = m.x;
    if (sigma) {
      const double var = (m.y - m.x * m.x / B) * (B / (B - 1.0));
      sigma[i] = var > 0.0 ? sqrt(var) : 0.0;
    }
  }
}

}  // namespace

cudaError_t launch_fold_moments(double *tally, double2 *mom, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_fold_moments<<<grid, 256, 0, s>>>(tally, mom, n);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_moment_read(const double2 *mom, double *total, double *sigma, int64_t n, double B,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_moment_read<<<grid, 256, 0, s>>>(mom, total, sigma, n, B);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ray_caps(const BoundGeom &g, const RayPtrs &rays, uint32_t *cap, int num_sms,
                            cudaStream_t s) {
  if (rays.n <= 0) return cudaSuccess;
  const int block = 256;
  const int grid = (int)std::min<int64_t>((rays.n + block - 1) / block, (int64_t)num_sms * 8);
  k_ray_caps<<<grid, block, 0, s>>>(g, rays, cap);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pair_fold(const PairOut &p, int64_t n_rays, int n_buckets, uint32_t *base, uint32_t *tiles,
                             ulonglong2 *sorted, double2 *mom, unsigned int *status, int num_sms,
                             cudaStream_t s) {
  if (n_rays <= 0) return cudaSuccess;
  cudaError_t e;
  const int grid = (int)std::min<int64_t>((n_rays + 255) / 256, (int64_t)num_sms * 8);
  // p.bcount[n_buckets] stays 0, so base[n_buckets] is the number of pairs
  if ((e = launch_exclusive_scan(p.bcount, (int64_t)n_buckets + 1, base, tiles, s)) != cudaSuccess) return e;
  // the scatter's cursors (in the count array) start at the bases
  if ((e = cudaMemcpyAsync(p.bcount, base, sizeof(uint32_t) * (size_t)n_buckets, cudaMemcpyDeviceToDevice, s)) !=
      cudaSuccess)
    return e;
  k_pair_scatter<<<grid, kFoldThreads, 0, s>>>(p, n_rays, p.bcount, sorted);
  const int fold_smem = 2 * 8 * kFoldSlots;
  if ((e = cudaFuncSetAttribute(k_pair_fold, cudaFuncAttributeMaxDynamicSharedMemorySize, fold_smem)) != cudaSuccess) return e;
  const int fgrid = (int)std::min<int64_t>(n_buckets, (int64_t)num_sms * kFoldBlocksPerSm);
  k_pair_fold<<<fgrid, kFoldBlockThreads, fold_smem, s>>>(sorted, base, n_buckets, mom, status);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace vrc
