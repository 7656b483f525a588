// vrc_sort_rays_static: the ray sort of vrc_cast_rays, for callers that must
// not allocate device memory once their run has started.
//
// Who needs it: a transport code that hands all free device memory to its
// own pool at start-up (a later cudaMalloc from a library would fail or
// fragment that pool), or one whose batch loop must not pay the implicit
// device-wide synchronisation of cudaMalloc / cudaFree while the CPU random
// walk keeps running.  vrc_cast_rays grows its sort scratch on demand; this
// entry point instead keeps the sort's scratch (keys, per-chunk key counts,
// write offsets, scan tile sums) in one file-scope device array of fixed size
// and allocates nothing.  The caller passes the input rays and the output
// array; both are device memory it owns.
#include <stdint.h>

#include <mutex>

#include "vrc.h"
#include "vrc_internal.h"
#include "vrc_sort.h"

namespace {

constexpr int64_t kMaxRays = (int64_t)1 << 18;  // rays per call
constexpr int64_t kMaxKeys = 16384;             // sort keys (groups x length buckets + 1)
constexpr int kMaxDevices = 64;
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Layout for the largest batch (chunks of 8,192 rays, 8,192-entry scan tiles).
constexpr int64_t kMaxChunks = (kMaxRays + 8191) / 8192;
constexpr size_t kKeysBytes = align_up(sizeof(uint32_t) * (size_t)kMaxRays);
constexpr size_t kTableBytes = align_up(sizeof(uint32_t) * (size_t)(kMaxKeys * kMaxChunks));
constexpr size_t kTilesBytes = align_up(sizeof(uint32_t) * (size_t)((kMaxKeys * kMaxChunks + 8191) / 8192));
constexpr size_t kScratchBytes = kKeysBytes + 2 * kTableBytes + kTilesBytes;  // about 5 MiB

// The scratch itself.  A device holds it from the moment this file's module
// is placed on that device (the first vrc_sort_rays_static call there, see
// scratch_address) until the process exits.  Host code must not use its
// name as an address.
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {};

// Set-up, once per device (`dev` must be current): the device address of
// g_sort_scratch, and the sort kernels made resident.  With CUDA's lazy
// module loading (the default since CUDA 12.2) a module reaches a device the
// first time one of its kernels or symbols is used there, and placing it can
// allocate device memory; doing both here, in the first call, means that
// later calls find everything in place and allocate nothing.
int scratch_address(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || p == nullptr)
      return vrc::set_last_error(VRC_ERR_CUDA, "cudaGetSymbolAddress of the static sort scratch failed");
    e = vrc::load_sort_kernels();
    if (e != cudaSuccess)
      return vrc::set_last_error(VRC_ERR_CUDA, "loading the sort kernels failed");
    g_scratch_dev[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_dev[dev];
  return VRC_OK;
}

}  // namespace

extern "C" int vrc_sort_rays_static(vrc_ctx *c, const vrc_rays *in, float *out, void *cuda_stream) {
  using namespace vrc;
  if (!c) return set_last_error(VRC_ERR_ARG, "context is NULL");
  if (!in || !out) return set_last_error(VRC_ERR_ARG, "rays or output is NULL");
  if (!in->on_device) return set_last_error(VRC_ERR_ARG, "vrc_sort_rays_static takes device rays only");
  if (in->n < 0) return set_last_error(VRC_ERR_ARG, "ray count is negative");
  if (in->n > kMaxRays)
    return set_last_error(VRC_ERR_ARG,
                          "vrc_sort_rays_static sorts at most 262144 rays per call (fixed 5 MiB "
                          "scratch); split the batch");
  if (in->n == 0) return VRC_OK;
  if (!in->x || !in->y || !in->z || !in->u || !in->v || !in->w || !in->E || !in->wt)
    return set_last_error(VRC_ERR_ARG, "a ray array is NULL");

  SortKeyArgs P;
  const double *edges = nullptr;
  int dev = 0;
  cudaStream_t ctx_stream = nullptr;
  ctx_sort_args(c, &P, &edges, &dev, &ctx_stream);
  if (P.n_keys > kMaxKeys) return set_last_error(VRC_ERR_ARG, "too many sort keys for the static scratch");
  if (dev < 0 || dev >= kMaxDevices) return set_last_error(VRC_ERR_ARG, "device ordinal out of range");

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return set_last_error(VRC_ERR_CUDA, "cudaGetDevice failed");
  if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
    return set_last_error(VRC_ERR_CUDA, "cannot select the context's device");
  unsigned char *base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc == VRC_OK) {
    const SortPlan plan = make_sort_plan(in->n, P.n_keys);
    if (plan.bytes_keys > kKeysBytes || plan.bytes_table > kTableBytes || plan.bytes_tiles > kTilesBytes) {
      rc = set_last_error(VRC_ERR_ARG, "batch does not fit the static sort scratch");
    } else {
      uint32_t *keys = reinterpret_cast<uint32_t *>(base);
      uint32_t *table = reinterpret_cast<uint32_t *>(base + kKeysBytes);
      uint32_t *offsets = reinterpret_cast<uint32_t *>(base + kKeysBytes + kTableBytes);
      uint32_t *tiles = reinterpret_cast<uint32_t *>(base + kKeysBytes + 2 * kTableBytes);
      const int64_t n = in->n;
      RayOut o = {out, out + n, out + 2 * n, out + 3 * n, out + 4 * n, out + 5 * n, out + 6 * n, out + 7 * n};
      RayPtrs rp;
      rp.aos = nullptr;
      rp.x = in->x; rp.y = in->y; rp.z = in->z; rp.u = in->u;
      rp.v = in->v; rp.w = in->w; rp.E = in->E; rp.wt = in->wt;
      rp.n = n;
      cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx_stream;
      cudaError_t e = launch_sort(rp, P, edges, plan, keys, table, offsets, tiles, o, s);
      if (e != cudaSuccess) rc = set_last_error(VRC_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return rc;
}
