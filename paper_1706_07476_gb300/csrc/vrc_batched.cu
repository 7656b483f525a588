// Batched form: many independent tally problems (each its own mesh, cross
// sections, rays and tally) cast by one persistent kernel.  Work items are
// chunks of one problem's rays; every block takes the next item from a
// global counter until the list is exhausted.  The per-ray code is the same
// as the single-problem kernel's (Sec. 3: lookup, cast, Eq. 4 score): cast_one,
// or in the plain form the warp-batched cast_one_plain_warp.
#include <algorithm>

#include "vrc_device.cuh"

namespace vrc {

namespace {

inline size_t align16(size_t x) { return (x + 15) / 16 * 16; }

struct BatchSmem {
  size_t hash, edges, sig, inv, queue, total;
};


BatchSmem batch_smem(int form, const BatchShape &sh, int block) {
  BatchSmem L;
  size_t off = 0;
  L.hash = off;
  off = align16(off + sizeof(int32_t) * ((size_t)sh.max_hash + 1));
  L.edges = off;
  off = align16(off + sizeof(double) * ((size_t)sh.max_groups + 1));
  L.sig = off;
  if (form == kFormPlain) {
    off = align16(off + sizeof(float) * (size_t)sh.max_mat * block);
    L.inv = off;
    off = align16(off + sizeof(double) * (size_t)sh.max_mat * block);
  } else {  // (sigma, 1/sigma) float pairs
    L.inv = off + sizeof(float);
    off = align16(off + 2 * sizeof(float) * (size_t)sh.max_mat * block);
  }
  L.queue = off;
  if (form == kFormPlain) off = align16(off + kWarpQueueBytes * (size_t)(block / 32));
  L.total = off;
  return L;
}

// CHUNKED: the block's warps take an item's rays rays_per_warp at a time from
// a shared counter; otherwise interleaved (a separate instantiation, so the
// default kernel's code is not changed by the option).
template <int FORM, bool CHUNKED>
__global__ void __launch_bounds__(256, FORM == kFormPlain ? 2 : 4)
    k_cast_batched(const CastArgs *__restrict__ probs, const BatchItem *__restrict__ items, int n_items,
                   unsigned int *queue, int rays_per_warp, BatchSmem L) {
  typedef typename Attenuation<FORM>::inv_t inv_t;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CastArgs A;
  __shared__ int s_item;
  __shared__ unsigned s_next;  // rays of the current item handed out (rays_per_warp > 0)
  int32_t *hash_s = reinterpret_cast<int32_t *>(smem + L.hash);
  double *edges_s = reinterpret_cast<double *>(smem + L.edges);
  const int lanes = FORM == kFormPlain ? 1 : 2;  // FP32: (sigma, 1/sigma) pairs
  float *sig_s = reinterpret_cast<float *>(smem + L.sig) + lanes * threadIdx.x;
  inv_t *inv_s = reinterpret_cast<inv_t *>(smem + L.inv) + lanes * threadIdx.x;
  const int stride = lanes * blockDim.x;
  int cur = -1;
  // Each pass takes one item index; indices only grow, so at most n_items passes.
  for (int pass = 0; pass < n_items; ++pass) {
    if (threadIdx.x == 0) {
      s_item = (int)atomicAdd(queue, 1u);
      s_next = 0;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    if (item.problem != cur) {  // block-uniform
      if (threadIdx.x == 0) A = probs[item.problem];
      __syncthreads();
      if (A.xs.n_union > 0)
        for (int t = threadIdx.x; t <= A.xs.n_hash; t += blockDim.x) hash_s[t] = A.xs.hash[t];
      if (A.edges)
        for (int t = threadIdx.x; t <= A.n_groups; t += blockDim.x) edges_s[t] = A.edges[t];
      __syncthreads();
      cur = item.problem;
    }
    const double *edges = A.edges ? edges_s : nullptr;
    RayCounts cnt;
    const int64_t end = item.start + item.count;
    if constexpr (CHUNKED) {  // rays_per_warp rays at a time from the item's counter
      const int lane = threadIdx.x & 31;
      for (;;) {
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(&s_next, (unsigned)rays_per_warp);
        c = __shfl_sync(0xffffffffu, c, 0);
        const int64_t first = item.start + (int64_t)c;
        if (first >= end) break;
        const int64_t stop = min(first + (int64_t)rays_per_warp, end);
        for (int64_t base = first; base < stop; base += 32) {
          if constexpr (FORM == kFormPlain) {  // warp-collective walk
            cast_one_plain_warp<false, TallyMaker, false>(A, base + lane, base + lane < stop, hash_s, edges,
                                                          sig_s, inv_s, stride, warp_queue(smem + L.queue), cnt);
          } else if (base + lane < stop) {
            cast_one<FORM>(A, base + lane, hash_s, edges, sig_s, inv_s, stride, cnt);
          }
        }
      }
    } else if constexpr (FORM == kFormPlain) {  // warp-collective walk: warp-uniform trip count
      const WarpQueue Q = warp_queue(smem + L.queue);
      const int lane = threadIdx.x & 31;
      for (int64_t base = item.start + (threadIdx.x & ~31); base < end; base += blockDim.x)
        cast_one_plain_warp<false, TallyMaker, false>(A, base + lane, base + lane < end, hash_s, edges,
                                                      sig_s, inv_s, stride, Q, cnt);
    } else {
      for (int64_t r = item.start + threadIdx.x; r < end; r += blockDim.x)
        cast_one<FORM>(A, r, hash_s, edges, sig_s, inv_s, stride, cnt);
    }
    flush_counts(cnt, A.counters, A.status);
    __syncthreads();  // s_item, A and the staged tables are reused next pass
  }
}

}  // namespace

size_t batched_smem_bytes(int form, const BatchShape &sh, int block) {
  return batch_smem(form, sh, block).total;
}

template <int FORM, bool CHUNKED>
cudaError_t set_smem(size_t smem) {
  return cudaFuncSetAttribute(k_cast_batched<FORM, CHUNKED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t batched_occupancy(int form, const BatchShape &sh, int block, int *blocks_per_sm) {
  const size_t smem = batched_smem_bytes(form, sh, block);
  cudaError_t e;
  if (form == kFormPlain) {
    if ((e = set_smem<kFormPlain, false>(smem)) != cudaSuccess || (e = set_smem<kFormPlain, true>(smem)) != cudaSuccess)
      return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_cast_batched<kFormPlain, false>, block, smem);
  }
  if ((e = set_smem<kFormFp32, false>(smem)) != cudaSuccess || (e = set_smem<kFormFp32, true>(smem)) != cudaSuccess)
    return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_cast_batched<kFormFp32, false>, block, smem);
}

cudaError_t launch_batched_cast(int form, const CastArgs *probs, const BatchItem *items, int n_items,
                                unsigned int *queue, const BatchShape &sh, int grid, int block,
                                int rays_per_warp, cudaStream_t s) {
  const BatchSmem L = batch_smem(form, sh, block);
  const bool chunked = rays_per_warp > 0;
  if (form == kFormPlain) {
    if (chunked)
      k_cast_batched<kFormPlain, true><<<grid, block, L.total, s>>>(probs, items, n_items, queue, rays_per_warp, L);
    else
      k_cast_batched<kFormPlain, false><<<grid, block, L.total, s>>>(probs, items, n_items, queue, 0, L);
  } else {
    if (chunked)
      k_cast_batched<kFormFp32, true><<<grid, block, L.total, s>>>(probs, items, n_items, queue, rays_per_warp, L);
    else
      k_cast_batched<kFormFp32, false><<<grid, block, L.total, s>>>(probs, items, n_items, queue, 0, L);
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace vrc
