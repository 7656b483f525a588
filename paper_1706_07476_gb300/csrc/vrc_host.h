// Host-side internals shared by the translation units of the libvrc C ABI
// (vrc_api*.cu): the context struct, error reporting, device and buffer
// helpers, and the cast steps that several entry points share.  Not part of
// the public ABI (include/vrc.h).
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vrc.h"
#include "vrc_internal.h"
#include "vrc_mlp.h"
#include "vrc_sort.h"

namespace vrc {
namespace host {

// Records the message for vrc_last_error and returns code.
int fail(int code, const char *fmt, ...);
// A CUDA error as VRC_ERR_OOM (allocation) or VRC_ERR_CUDA.
int cuda_fail(cudaError_t e, const char *what);
// Process-wide count of launched kernels (vrc_launch_count).
extern std::atomic<long long> g_launches;

// Every device and pinned-host allocation of the library goes through these
// two, so that vrc_debug_fail_alloc can make a chosen one fail (with
// cudaErrorMemoryAllocation, before the driver is asked) and tests can walk
// each failure path without exhausting a GPU.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t pinned_alloc(void **p, size_t bytes);

#define VRC_CUDA(call, what)                            \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
  } while (0)

// Sets a device for the scope of an API call and restores the previous one.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Grow-only device buffer.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t want) {
    if (want <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = dev_malloc(&p, want);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

inline df split(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return {hi, lo};
}

inline bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// A pair of events bracketing one group of kernel launches.
struct TimedSpan {
  cudaEvent_t start, stop;
  int kind;  // 0 cast, 1 sort
};

}  // namespace host
}  // namespace vrc

using vrc::host::DevBuf;
using vrc::host::DeviceGuard;
using vrc::host::TimedSpan;

struct vrc_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  vrc_options opt;
  int32_t n[3] = {0, 0, 0};
  double org[3] = {0, 0, 0}, h[3] = {0, 0, 0};  // rectilinear: first plane, mean spacing
  bool rect = false;
  DevBuf rectDf;     // plane positions as (hi, lo) float pairs, x then y then z
  DevBuf rectD;      // plane positions, float64, same order
  DevBuf rectWidth;  // cell widths, float64, x then y then z
  int64_t rect_off[3] = {0, 0, 0};  // first plane of each axis in rectDf / rectD
  int64_t ncells = 0;
  int32_t n_materials = 0, n_groups = 1;
  std::vector<double> edges;
  std::vector<uint8_t> used;
  std::vector<std::vector<double>> tabE, tabS;
  std::vector<uint8_t> loaded;
  bool xs_dirty = true;

  uint8_t *d_mat = nullptr;
  double *d_edges = nullptr;
  double *d_tally = nullptr;
  unsigned long long *d_counters = nullptr;
  unsigned int *d_status = nullptr;
  unsigned long long *d_queue = nullptr;  // ray counter of a cast with rays_per_warp > 0

  int32_t n_union = 0, m_pad = 0, n_hash = 0;
  float l2min = 0.f, inv_bw = 0.f;
  DevBuf xsE, xsInvdE, xsS, xsHash;
  DevBuf stage;    // device copy of host rays
  // pipelined upload of large host batches: a copy stream, two staging slots
  // of one chunk each, and per slot an event after its upload and one after
  // the cast that reads it
  cudaStream_t up_stream = nullptr;
  DevBuf up_slot[2];
  cudaEvent_t up_copied[2] = {nullptr, nullptr}, up_freed[2] = {nullptr, nullptr};
  DevBuf scratch;  // finalize staging
  DevBuf sortKeys, sortTable, sortOffsets, sortTiles, sortRays;  // ray-sort scratch
  int xs_mode = VRC_XS_TABLE;
  bool mlp_ready = false;
  uint32_t mlp_mask = 0;          // outputs the surrogate models (non-void materials)
  double mlp_lo = 0, mlp_hi = 0;  // energy range of the tables
  DevBuf mlpParams, mlpFlags, sigBuf;
  DevBuf mom;  // moments of the tally: (S1, S2) per (group, cell), sums of samples and of their squares
  DevBuf detPos, detOut;  // next-event detectors and their flux
  bool moments = false;
  int moment_mode = VRC_MOMENTS_OFF;
  int64_t batches = 0;    // samples folded into the moments (batches or histories)
  DevBuf pairBuf;         // per-history cast: (key, score) pairs, each ray's stretch
  DevBuf pairSorted;      // the pairs sorted into bin buckets
  DevBuf rayCap, rayOff, rayCnt;  // per ray: room, first pair, pairs written (uint32)
  DevBuf pairBoff, pairTiles;  // bucket counts (then cursors) and bases; scan scratch
  DevBuf histIds;         // device copy of host history ids
  DevBuf histSorted;      // history ids in sorted ray order
  DevBuf histBound;       // last room and last offset of the current call (pair count)

  bool timing = false;
  std::vector<TimedSpan> pending;
  std::vector<cudaEvent_t> event_pool;
  double cast_ms = 0.0, sort_ms = 0.0;
  int64_t cast_launches = 0;

  cudaError_t get_event(cudaEvent_t *e) {
    if (!event_pool.empty()) {
      *e = event_pool.back();
      event_pool.pop_back();
      return cudaSuccess;
    }
    return cudaEventCreate(e);
  }

  ~vrc_ctx() {
    DeviceGuard g(device);
    if (stream) cudaStreamSynchronize(stream);
    if (up_stream) cudaStreamSynchronize(up_stream);
    for (int i = 0; i < 2; ++i) {
      if (up_copied[i]) cudaEventDestroy(up_copied[i]);
      if (up_freed[i]) cudaEventDestroy(up_freed[i]);
      up_slot[i].release();
    }
    if (up_stream) cudaStreamDestroy(up_stream);
    for (auto &t : pending) {
      cudaEventSynchronize(t.stop);
      cudaEventDestroy(t.start);
      cudaEventDestroy(t.stop);
    }
    for (auto e : event_pool) cudaEventDestroy(e);
    cudaFree(d_mat);
    cudaFree(d_edges);
    cudaFree(d_tally);
    cudaFree(d_counters);
    cudaFree(d_status);
    cudaFree(d_queue);
    xsE.release();
    xsInvdE.release();
    xsS.release();
    xsHash.release();
    stage.release();
    scratch.release();
    sortKeys.release();
    sortTable.release();
    sortOffsets.release();
    sortTiles.release();
    sortRays.release();
    mlpParams.release();
    mlpFlags.release();
    sigBuf.release();
    mom.release();
    pairBuf.release();
    pairSorted.release();
    rayCap.release();
    rayOff.release();
    rayCnt.release();
    pairBoff.release();
    pairTiles.release();
    histIds.release();
    histSorted.release();
    histBound.release();
    rectDf.release();
    rectD.release();
    rectWidth.release();
    detPos.release();
    detOut.release();
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace vrc {
namespace host {

int check_options(const vrc_options *o);
// Builds the union energy grid, the per-material sigma rows on it, the
// interval reciprocals and the log2 hash, and uploads them.
int build_xs(vrc_ctx *c);
// Kernel arguments of a cast of rays on this context.
CastArgs make_args(const vrc_ctx *c, const RayPtrs &rays);
// The status word's bits as an error code (with its message).
int status_code(unsigned st);
// Waits for the caller's stream (if any) and the context's stream.
int sync_streams(vrc_ctx *c, void *stream);
// Batches of at least this many rays are sorted when options.sort is -1.
constexpr int64_t kAutoSortMin = 65536;
// Crossed-cell buckets per group of the sort key when options.sort_len_buckets
// is -1 (halved while groups x buckets + 1 would pass the key limit).
// slab256, chunks of 32 rays per warp: 256 buckets 16.9 ms (FP32) and 44.7 ms
// (plain) per sort and cast, 64 buckets 17.0 and 45.0 ms.
constexpr int kAutoLenBuckets = 256;
// FP32 casts of at least this many rays hand rays to warps in chunks of 32
// from a counter when options.rays_per_warp is 0 (auto).
constexpr int64_t kAutoChunkMinRays = (int64_t)1 << 23;
// Sorts the batch into context scratch and points rp at the sorted copy.
// When carry_out is set, carry_in[i] (one uint32 per ray) goes to the sorted
// position of ray i.
// With spatial set, the key is (group, spatial block of the start point)
// instead, for point events (the direction is not used).
// With n_accepted set, rays in the learned surrogate's accepted energy bins
// are put first and *n_accepted receives the device address of their count.
int sort_rays(vrc_ctx *c, RayPtrs &rp, cudaStream_t s, const uint32_t *carry_in = nullptr,
              uint32_t *carry_out = nullptr, bool spatial = false,
              const uint32_t **n_accepted = nullptr);
// Sort (optional), surrogate (optional) and cast of a device batch on stream s.
int cast_device(vrc_ctx *c, RayPtrs rp, cudaStream_t s);
// Device view of a ray batch: device arrays as given, host arrays copied
// into the context's staging buffer on stream s.
int ray_ptrs(vrc_ctx *c, const vrc_rays *r, cudaStream_t s, RayPtrs *out);

}  // namespace host
}  // namespace vrc
