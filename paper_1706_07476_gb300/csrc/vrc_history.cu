// Tally moments (the sums behind the tally's standard deviation in Eqs. 5
// and 8), kept as (S1, S2) pairs per (group, cell): the batch fold, the read
// (S1 and sigma), and for per-history moments the segment bound that sizes
// the history table and the drain that turns the table's per-(history,
// cell) sums x into S1 += x, S2 += x^2.
#include <algorithm>
#include <math.h>

#include "vrc_internal.h"

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

__global__ void k_segment_bound(BoundGeom G, RayPtrs R, unsigned long long *bound) {
  unsigned long long acc = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R.n;
       r += (int64_t)gridDim.x * blockDim.x) {
    float f[6];
    if (R.aos) {
      const float4 a = R.aos[2 * r], b = R.aos[2 * r + 1];
      f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y;
    } else {
      f[0] = R.x[r]; f[1] = R.y[r]; f[2] = R.z[r]; f[3] = R.u[r]; f[4] = R.v[r]; f[5] = R.w[r];
    }
    acc += ray_bound(G, f);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(bound, acc);
}

// Every claimed slot (key + 1, x), found from the bitmap: mom[bin] += (x,
// x^2), slot = 0, bitmap word = 0.  S1 and S2 of a bin share a 16-byte pair,
// so the two reductions of a slot touch one 32-byte sector: one DRAM
// read-modify-write where separate S1 and S2 arrays took two.
__global__ void k_hist_drain(ulonglong2 *e, unsigned int *bits, unsigned long long words,
                             double2 *__restrict__ mom) {
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < words;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned w = bits[j];
    if (w == 0u) continue;
    bits[j] = 0u;
    while (w) {
      const int b = __ffs(w) - 1;
      w &= w - 1u;
      ulonglong2 *slot = e + 32ull * j + (unsigned)b;
      const ulonglong2 v = *slot;
      const unsigned bin = (unsigned)((v.x - 1ull) & 0xffffffffull);
      const double x = __longlong_as_double((long long)v.y);
      atomicAdd(&mom[bin].x, x);
      atomicAdd(&mom[bin].y, x * x);
      *slot = make_ulonglong2(0ull, 0ull);
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

cudaError_t launch_segment_bound(const BoundGeom &g, const RayPtrs &rays, unsigned long long *bound,
                                 int num_sms, cudaStream_t s) {
  if (rays.n <= 0) return cudaSuccess;
  const int block = 256;
  const int grid = (int)std::min<int64_t>((rays.n + block - 1) / block, (int64_t)num_sms * 8);
  k_segment_bound<<<grid, block, 0, s>>>(g, rays, bound);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_hist_drain(const HistTable &t, double2 *mom, int num_sms, cudaStream_t s) {
  const unsigned long long words = (t.mask + 1ull) / 32ull;
  const int block = 256;
  const int grid = (int)std::min<unsigned long long>((words + block - 1) / block, (unsigned long long)num_sms * 8);
  k_hist_drain<<<grid, block, 0, s>>>(reinterpret_cast<ulonglong2 *>(t.e), t.bits, words, mom);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace vrc
