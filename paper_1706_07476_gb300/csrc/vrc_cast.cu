// The VRC cast kernel (Sec. 3: one GPU thread per ray runs the cross-section
// lookup, the ray cast and the VRC score of Eq. 4) and the tally finalize
// kernel.
#include <algorithm>
#include <type_traits>

#include "vrc_device.cuh"

namespace vrc {

namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct SmemLayout {
  size_t hash, edges, sig, inv, queue, total;
};


SmemLayout smem_layout(int form, const CastArgs &a, int block) {
  SmemLayout L;
  size_t off = 0;
  L.hash = off;
  off += sizeof(int32_t) * (a.xs.n_union > 0 ? (size_t)a.xs.n_hash + 1 : 1);
  off = align_up(off, 16);
  L.edges = off;
  off += sizeof(double) * (a.edges ? (size_t)a.n_groups + 1 : 1);
  off = align_up(off, 16);
  L.sig = off;
  if (form == kFormPlain) {  // float sigma [M][B], then double 1/sigma [M][B]
    off += sizeof(float) * (size_t)a.xs.n_mat * block;
    off = align_up(off, 16);
    L.inv = off;
    off += sizeof(double) * (size_t)a.xs.n_mat * block;
  } else {  // (sigma, 1/sigma) float pairs [M][B]
    L.inv = off + sizeof(float);
    off += 2 * sizeof(float) * (size_t)a.xs.n_mat * block;
  }
  off = align_up(off, 16);
  L.queue = off;
  if (form == kFormPlain) off += kWarpQueueBytes * (size_t)(block / 32);
  L.total = align_up(off, 16);
  return L;
}

// Blocks per SM: 2 for the plain form (its warp queues and float64 state),
// 4 for the FP32 form.
template <int FORM, bool SURR, typename Maker = TallyMaker, bool RECT = false>
__global__ void __launch_bounds__(256, FORM == kFormPlain ? 2 : 4)
    k_cast(CastArgs a, SmemLayout L) {
  typedef typename Attenuation<FORM>::inv_t inv_t;
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *hash_s = reinterpret_cast<int32_t *>(smem + L.hash);
  double *edges_s = reinterpret_cast<double *>(smem + L.edges);
  const int lanes = FORM == kFormPlain ? 1 : 2;  // FP32: (sigma, 1/sigma) pairs
  float *sig_s = reinterpret_cast<float *>(smem + L.sig) + lanes * threadIdx.x;
  inv_t *inv_s = reinterpret_cast<inv_t *>(smem + L.inv) + lanes * threadIdx.x;

  if (a.xs.n_union > 0)
    for (int t = threadIdx.x; t <= a.xs.n_hash; t += blockDim.x) hash_s[t] = a.xs.hash[t];
  if (a.edges)
    for (int t = threadIdx.x; t <= a.n_groups; t += blockDim.x) edges_s[t] = a.edges[t];
  __syncthreads();
  const double *edges = a.edges ? edges_s : nullptr;
  const int stride = lanes * blockDim.x;

  RayCounts cnt;
  const int lane = threadIdx.x & 31;
  // one round: the 32 rays base + lane of this warp (warp-uniform base)
  auto round = [&](int64_t base) {
    if constexpr (FORM == kFormPlain) {  // the batched walk is warp-collective
      cast_one_plain_warp<SURR, Maker, RECT>(a, base + lane, base + lane < a.rays.n, hash_s, edges,
                                             sig_s, inv_s, stride, warp_queue(smem + L.queue), cnt);
    } else if (base + lane < a.rays.n) {
      cast_one<FORM, SURR, Maker, RECT>(a, base + lane, hash_s, edges, sig_s, inv_s, stride, cnt);
    }
  };
  if (a.rays_per_warp > 0) {
    // dynamic: the warp takes rays_per_warp consecutive rays at a time from
    // the launch's counter (the counter only grows, so the loop ends)
    const unsigned long long n = (unsigned long long)a.rays.n;
    for (;;) {
      unsigned long long first = 0;
      if (lane == 0) first = atomicAdd(a.queue, (unsigned long long)a.rays_per_warp);
      first = __shfl_sync(0xffffffffu, first, 0);
      if (first >= n) break;
      const int64_t end = (int64_t)min(first + (unsigned long long)a.rays_per_warp, n);
      for (int64_t base = (int64_t)first; base < end; base += 32) round(base);
    }
  } else {
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.rays.n;
         base += (int64_t)gridDim.x * blockDim.x)
      round(base);
  }
  flush_counts(cnt, a.counters, a.status);
}

__global__ void k_scale_copy(const double *__restrict__ src, double *__restrict__ dst, int64_t n,
                             double scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] * scale;
}

}  // namespace

size_t cast_smem_bytes(int form, const CastArgs &a, int block) {
  return smem_layout(form, a, block).total;
}

template <int FORM, bool SURR, typename Maker, bool RECT>
cudaError_t occupancy_r(const CastArgs &a, int block, int *bps) {
  const size_t smem = cast_smem_bytes(FORM, a, block);
  cudaError_t e = cudaFuncSetAttribute(k_cast<FORM, SURR, Maker, RECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_cast<FORM, SURR, Maker, RECT>, block, smem);
}

template <int FORM, bool SURR, typename Maker, bool RECT>
cudaError_t launch_r(const CastArgs &a, int grid, int block, cudaStream_t s) {
  const SmemLayout L = smem_layout(FORM, a, block);
  cudaError_t e = cudaFuncSetAttribute(k_cast<FORM, SURR, Maker, RECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e != cudaSuccess) return e;
  k_cast<FORM, SURR, Maker, RECT><<<grid, block, L.total, s>>>(a, L);
  note_launches(1);
  return cudaGetLastError();
}

// uniform or rectilinear mesh, chosen by the mesh descriptor
template <int FORM, bool SURR, typename Maker = TallyMaker>
cudaError_t occupancy_t(const CastArgs &a, int block, int *bps) {
  return a.mesh.rect ? occupancy_r<FORM, SURR, Maker, true>(a, block, bps)
                     : occupancy_r<FORM, SURR, Maker, false>(a, block, bps);
}

template <int FORM, bool SURR, typename Maker = TallyMaker>
cudaError_t launch_t(const CastArgs &a, int grid, int block, cudaStream_t s) {
  return a.mesh.rect ? launch_r<FORM, SURR, Maker, true>(a, grid, block, s)
                     : launch_r<FORM, SURR, Maker, false>(a, grid, block, s);
}

cudaError_t cast_occupancy(int form, const CastArgs &a, int block, int *blocks_per_sm) {
  const bool surr = a.sig_ray != nullptr;
  if (form == kFormPlain)
    return surr ? occupancy_t<kFormPlain, true>(a, block, blocks_per_sm) : occupancy_t<kFormPlain, false>(a, block, blocks_per_sm);
  return surr ? occupancy_t<kFormFp32, true>(a, block, blocks_per_sm) : occupancy_t<kFormFp32, false>(a, block, blocks_per_sm);
}

cudaError_t launch_cast(int form, const CastArgs &a, int grid, int block, cudaStream_t s) {
  const bool surr = a.sig_ray != nullptr;
  if (form == kFormPlain)
    return surr ? launch_t<kFormPlain, true>(a, grid, block, s) : launch_t<kFormPlain, false>(a, grid, block, s);
  return surr ? launch_t<kFormFp32, true>(a, grid, block, s) : launch_t<kFormFp32, false>(a, grid, block, s);
}

// Per-history cast: the same kernel with each ray's pair stretch as the
// sink (tabulated cross sections; the ray order is the caller's).
cudaError_t cast_hist_occupancy(int form, const CastArgs &a, int block, int *blocks_per_sm) {
  if (form == kFormPlain) return occupancy_t<kFormPlain, false, PairMaker>(a, block, blocks_per_sm);
  return occupancy_t<kFormFp32, false, PairMaker>(a, block, blocks_per_sm);
}

cudaError_t launch_cast_hist(int form, const CastArgs &a, int grid, int block, cudaStream_t s) {
  if (form == kFormPlain) return launch_t<kFormPlain, false, PairMaker>(a, grid, block, s);
  return launch_t<kFormFp32, false, PairMaker>(a, grid, block, s);
}

namespace {
__global__ void k_per_volume_rect(const double *__restrict__ src, double *__restrict__ dst, int64_t n,
                                  int64_t first, int32_t nx, int32_t ny, int64_t ncells,
                                  const double *__restrict__ wx, const double *__restrict__ wy,
                                  const double *__restrict__ wz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = (first + i) % ncells;
    const int64_t ix = cell % nx, iy = (cell / nx) % ny, iz = cell / ((int64_t)nx * ny);
    dst[i] = src[i] / (wx[ix] * wy[iy] * wz[iz]);
  }
}
}  // namespace

cudaError_t launch_per_volume_rect(const double *src, double *dst, int64_t n, int64_t first, int32_t nx,
                                   int32_t ny, int64_t ncells, const double *wx, const double *wy,
                                   const double *wz, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_per_volume_rect<<<grid, 256, 0, s>>>(src, dst, n, first, nx, ny, ncells, wx, wy, wz);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(const double *src, double *dst, int64_t n, double scale,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int block = 256;
  int64_t want = (n + block - 1) / block;
  int grid = (int)std::min<int64_t>(want, 152 * 8);
  k_scale_copy<<<grid, block, 0, s>>>(src, dst, n, scale);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace vrc
