// Host implementation of the libvrc C ABI (include/vrc.h).
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

using namespace vrc;

namespace {

thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(VRC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(VRC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

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
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

df split(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return {hi, lo};
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

void vrc::note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// A pair of events bracketing one group of kernel launches.
struct TimedSpan {
  cudaEvent_t start, stop;
  int kind;  // 0 cast, 1 sort
};

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
  DevBuf momS1, momS2;  // moments of the tally: sums of samples and of their squares
  DevBuf detPos, detOut;  // next-event detectors and their flux
  bool moments = false;
  int moment_mode = VRC_MOMENTS_OFF;
  int64_t batches = 0;    // samples folded into the moments (batches or histories)
  DevBuf histTab;         // per-history table, histCap slots of 16 bytes, all zero between calls
  unsigned long long histCap = 0;
  DevBuf histIds;         // device copy of host history ids
  DevBuf histSorted;      // history ids in sorted ray order
  DevBuf histBits;        // claim bitmap of the table, histCap bits, all zero between calls
  DevBuf histBound;       // segment bound of the current call

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
    momS1.release();
    momS2.release();
    histTab.release();
    histIds.release();
    histSorted.release();
    histBits.release();
    histBound.release();
    rectDf.release();
    rectD.release();
    rectWidth.release();
    detPos.release();
    detOut.release();
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

int check_options(const vrc_options *o) {
  if (o->form != VRC_FORM_PLAIN && o->form != VRC_FORM_FP32)
    return fail(VRC_ERR_ARG, "options.form must be VRC_FORM_PLAIN or VRC_FORM_FP32");
  if (o->block < 0 || o->block > 256 || (o->block % 32) != 0)
    return fail(VRC_ERR_ARG, "options.block must be 0 or a multiple of 32 up to 256");
  if (o->blocks_per_sm < 0) return fail(VRC_ERR_ARG, "options.blocks_per_sm must be >= 0");
  if (o->sort < -1 || o->sort > 1) return fail(VRC_ERR_ARG, "options.sort must be -1, 0 or 1");
  if (o->sort_len_buckets != -1 && (o->sort_len_buckets < 1 || o->sort_len_buckets > 256))
    return fail(VRC_ERR_ARG, "options.sort_len_buckets must be -1 or 1..256");
  if (o->stop_at_zero != 0 && o->stop_at_zero != 1) return fail(VRC_ERR_ARG, "options.stop_at_zero must be 0 or 1");
  return VRC_OK;
}

// Builds the union energy grid, the per-material sigma rows on it, the
// interval reciprocals and the log2 hash, and uploads them.
int build_xs(vrc_ctx *c) {
  for (int m = 0; m < c->n_materials; ++m)
    if (c->used[m] && !c->loaded[m])
      return fail(VRC_ERR_STATE, "material %d is used by the mesh but has no cross sections", m);
  std::vector<double> U;
  for (int m = 0; m < c->n_materials; ++m)
    if (c->loaded[m]) U.insert(U.end(), c->tabE[m].begin(), c->tabE[m].end());
  std::sort(U.begin(), U.end());
  U.erase(std::unique(U.begin(), U.end()), U.end());
  const int64_t nu = (int64_t)U.size();
  if (nu > (int64_t)1 << 30) return fail(VRC_ERR_ARG, "union energy grid too large");
  c->n_union = (int32_t)nu;
  c->m_pad = (c->n_materials + 3) & ~3;
  c->xs_dirty = false;
  if (nu == 0) return VRC_OK;

  std::vector<float> S((size_t)nu * c->m_pad, 0.f);
  for (int m = 0; m < c->n_materials; ++m) {
    const std::vector<double> &E = c->tabE[m], &Sg = c->tabS[m];
    const size_t n = E.size();
    if (!c->loaded[m] || n == 0) continue;
    size_t k = 0;
    for (int64_t i = 0; i < nu; ++i) {
      const double e = U[i];
      double s;
      if (n == 1 || e <= E[0]) s = Sg[0];
      else if (e >= E[n - 1]) s = Sg[n - 1];
      else {
        while (k + 1 < n && E[k + 1] <= e) ++k;  // E[k] <= e < E[k+1]
        s = Sg[k] + (e - E[k]) * (Sg[k + 1] - Sg[k]) / (E[k + 1] - E[k]);
      }
      S[(size_t)i * c->m_pad + m] = (float)s;
    }
  }
  std::vector<double> inv((size_t)std::max<int64_t>(nu - 1, 1), 0.0);
  for (int64_t i = 0; i + 1 < nu; ++i) inv[i] = 1.0 / (U[i + 1] - U[i]);

  int nh = 64;
  while (nh < 4096 && nh * 4 < nu) nh <<= 1;
  c->n_hash = nh;
  const double l2a = std::log2(U[0]), l2b = std::log2(U[nu - 1]);
  c->l2min = (float)l2a;
  c->inv_bw = l2b > l2a ? (float)(nh / (l2b - l2a)) : 0.f;
  std::vector<int32_t> hash((size_t)nh + 1);
  {
    int64_t i = 0;
    for (int b = 0; b <= nh; ++b) {
      double eb = (c->inv_bw > 0.f) ? std::exp2(l2a + b / (double)c->inv_bw) : U[0];
      while (i + 1 < nu && U[i + 1] <= eb) ++i;
      hash[b] = (int32_t)std::min<int64_t>(i, std::max<int64_t>(nu - 2, 0));
    }
  }
  VRC_CUDA(c->xsE.ensure(sizeof(double) * nu), "allocating the energy grid");
  VRC_CUDA(c->xsInvdE.ensure(sizeof(double) * inv.size()), "allocating the energy grid");
  VRC_CUDA(c->xsS.ensure(sizeof(float) * S.size()), "allocating the cross-section table");
  VRC_CUDA(c->xsHash.ensure(sizeof(int32_t) * hash.size()), "allocating the energy hash");
  VRC_CUDA(cudaStreamSynchronize(c->stream), "synchronizing before a table upload");
  VRC_CUDA(cudaMemcpy(c->xsE.p, U.data(), sizeof(double) * nu, cudaMemcpyHostToDevice), "uploading the energy grid");
  VRC_CUDA(cudaMemcpy(c->xsInvdE.p, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice), "uploading the energy grid");
  VRC_CUDA(cudaMemcpy(c->xsS.p, S.data(), sizeof(float) * S.size(), cudaMemcpyHostToDevice), "uploading the cross sections");
  VRC_CUDA(cudaMemcpy(c->xsHash.p, hash.data(), sizeof(int32_t) * hash.size(), cudaMemcpyHostToDevice), "uploading the energy hash");
  return VRC_OK;
}

CastArgs make_args(const vrc_ctx *c, const RayPtrs &rays) {
  CastArgs a;
  std::memset(&a, 0, sizeof a);
  for (int k = 0; k < 3; ++k) {
    a.mesh.n[k] = c->n[k];
    a.mesh.org[k] = split(c->org[k]);
    a.mesh.h[k] = split(c->h[k]);
    a.mesh.inv_h[k] = split(1.0 / c->h[k]);
  }
  a.mesh.stride[0] = 1;
  a.mesh.stride[1] = c->n[0];
  a.mesh.stride[2] = (int64_t)c->n[0] * c->n[1];
  a.mesh.ncells = c->ncells;
  a.mesh.mat = c->d_mat;
  if (c->rect) {
    a.mesh.rect = 1;
    for (int k = 0; k < 3; ++k) a.mesh.edge[k] = static_cast<const float2 *>(c->rectDf.p) + c->rect_off[k];
  }
  a.xs.n_union = c->n_union;
  a.xs.m_pad = c->m_pad;
  a.xs.n_mat = c->n_materials;
  a.xs.n_hash = c->n_hash;
  a.xs.l2min = c->l2min;
  a.xs.inv_bw = c->inv_bw;
  a.xs.E = static_cast<const double *>(c->xsE.p);
  a.xs.inv_dE = static_cast<const double *>(c->xsInvdE.p);
  a.xs.S = static_cast<const float *>(c->xsS.p);
  a.xs.hash = static_cast<const int32_t *>(c->xsHash.p);
  a.edges = c->edges.empty() ? nullptr : c->d_edges;
  a.n_groups = c->n_groups;
  a.rays = rays;
  a.tally = c->d_tally;
  a.stop_zero = c->opt.stop_at_zero;
  a.counters = c->d_counters;
  a.status = c->d_status;
  return a;
}

int status_code(unsigned st) {
  if (st & kStatusTimeout)
    return fail(VRC_ERR_CUDA, "a bounded wait on the tensor cores gave up; results are incomplete");
  if (st & kStatusTableFull)
    return fail(VRC_ERR_OOM, "the per-history table overflowed; its scores are incomplete");
  if (st & kStatusTraversal)
    return fail(VRC_ERR_TRAVERSAL, "a ray needed more grid steps than the mesh allows");
  if (st & kStatusNonfinite)
    return fail(VRC_ERR_NONFINITE,
                "a ray had a non-finite field, a non-positive energy or a zero direction");
  return VRC_OK;
}

int sync_streams(vrc_ctx *c, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (s && s != c->stream) VRC_CUDA(cudaStreamSynchronize(s), "synchronizing the caller's stream");
  VRC_CUDA(cudaStreamSynchronize(c->stream), "synchronizing the context stream");
  return VRC_OK;
}

constexpr int64_t kAutoSortMin = 65536;

// Sorts the batch into context scratch and points rp at the sorted copy.
// When carry_out is set, carry_in[i] (one uint32 per ray) goes to the sorted
// position of ray i.
int sort_rays(vrc_ctx *c, RayPtrs &rp, cudaStream_t s, const uint32_t *carry_in = nullptr,
              uint32_t *carry_out = nullptr) {
  SortKeyArgs P;
  std::memset(&P, 0, sizeof P);
  for (int k = 0; k < 3; ++k) {
    P.lo[k] = (float)c->org[k];
    P.hi[k] = (float)(c->org[k] + c->n[k] * c->h[k]);
    P.inv_h[k] = (float)(1.0 / c->h[k]);
    P.n[k] = c->n[k];
  }
  P.n_groups = c->n_groups;
  int nl = c->opt.sort_len_buckets > 0 ? c->opt.sort_len_buckets : 64;
  while (nl > 1 && (int64_t)c->n_groups * nl + 1 > 16384) nl >>= 1;
  P.n_len = nl;
  const int max_cells = c->n[0] + c->n[1] + c->n[2] + 1;
  P.len_width = std::max(1, (max_cells + nl - 1) / nl);
  P.n_keys = c->n_groups * nl + 1;
  SortPlan plan = make_sort_plan(rp.n, P.n_keys);
  VRC_CUDA(c->sortKeys.ensure(plan.bytes_keys), "allocating sort scratch");
  VRC_CUDA(c->sortTable.ensure(plan.bytes_table), "allocating sort scratch");
  VRC_CUDA(c->sortOffsets.ensure(plan.bytes_table), "allocating sort scratch");
  VRC_CUDA(c->sortTiles.ensure(plan.bytes_tiles), "allocating sort scratch");
  VRC_CUDA(c->sortRays.ensure(plan.bytes_rays), "allocating sort scratch");
  RayOut out;
  std::memset(&out, 0, sizeof out);
  out.aos = static_cast<float4 *>(c->sortRays.p);  // sorted copy as 32-byte records
  out.carry_in = carry_in;
  out.carry_out = carry_out;
  TimedSpan span{nullptr, nullptr, 1};
  if (c->timing) {
    VRC_CUDA(c->get_event(&span.start), "creating a timing event");
    VRC_CUDA(c->get_event(&span.stop), "creating a timing event");
    VRC_CUDA(cudaEventRecord(span.start, s), "recording a timing event");
  }
  VRC_CUDA(launch_sort(rp, P, c->edges.empty() ? nullptr : c->d_edges, plan,
                       static_cast<uint32_t *>(c->sortKeys.p), static_cast<uint32_t *>(c->sortTable.p),
                       static_cast<uint32_t *>(c->sortOffsets.p), static_cast<uint32_t *>(c->sortTiles.p),
                       out, s),
           "launching the ray sort");
  if (c->timing) {
    VRC_CUDA(cudaEventRecord(span.stop, s), "recording a timing event");
    c->pending.push_back(span);
  }
  rp.x = rp.y = rp.z = rp.u = rp.v = rp.w = rp.E = rp.wt = nullptr;
  rp.aos = out.aos;
  return VRC_OK;
}

// Sort (optional), surrogate (optional) and cast of a device batch on stream s.
int cast_device(vrc_ctx *c, RayPtrs rp, cudaStream_t s) {
  const bool do_sort = c->opt.sort == 1 || (c->opt.sort == -1 && rp.n >= kAutoSortMin);
  if (do_sort) {
    int rc = sort_rays(c, rp, s);
    if (rc) return rc;
  }
  const float *sig_ray = nullptr;
  if (c->xs_mode == VRC_XS_SURROGATE && c->mlp_ready) {
    VRC_CUDA(c->sigBuf.ensure(sizeof(float) * 16 * (size_t)rp.n), "allocating surrogate scratch");
    mlp::ApplyArgs aa;
    std::memset(&aa, 0, sizeof aa);
    aa.params = static_cast<const float *>(c->mlpParams.p);
    aa.E = rp.E;
    aa.aos = rp.aos;
    aa.n = rp.n;
    aa.out = static_cast<float *>(c->sigBuf.p);
    aa.mode = 1;
    aa.mat_mask = c->mlp_mask;
    aa.flags = static_cast<const uint8_t *>(c->mlpFlags.p);
    aa.n_hash = c->n_hash;
    aa.l2min = c->l2min;
    aa.inv_bw = c->inv_bw;
    aa.e_first = c->mlp_lo;
    aa.e_last = c->mlp_hi;
    aa.emb = mlp::make_embed(c->mlp_lo, c->mlp_hi);
    aa.status = c->d_status;
    VRC_CUDA(mlp::launch_apply(aa, c->num_sms, s), "launching the surrogate");
    sig_ray = aa.out;
  }
  CastArgs a = make_args(c, rp);
  a.sig_ray = sig_ray;
  const int form = c->opt.form;
  const int block = c->opt.block > 0 ? c->opt.block : 256;
  int bps = c->opt.blocks_per_sm;
  if (bps <= 0) {
    VRC_CUDA(cast_occupancy(form, a, block, &bps), "querying occupancy");
    if (bps <= 0) return fail(VRC_ERR_ARG, "cast kernel does not fit on an SM with %d materials", c->n_materials);
  }
  const int64_t need = (rp.n + block - 1) / block;
  const int grid = (int)std::min<int64_t>(need, (int64_t)c->num_sms * bps);
  TimedSpan span{nullptr, nullptr, 0};
  if (c->timing) {
    VRC_CUDA(c->get_event(&span.start), "creating a timing event");
    VRC_CUDA(c->get_event(&span.stop), "creating a timing event");
    VRC_CUDA(cudaEventRecord(span.start, s), "recording a timing event");
  }
  VRC_CUDA(launch_cast(form, a, grid, block, s), "launching the cast kernel");
  if (c->timing) {
    VRC_CUDA(cudaEventRecord(span.stop, s), "recording a timing event");
    c->pending.push_back(span);
    c->cast_launches += 1;
  }
  return VRC_OK;
}

// Device view of a ray batch: device arrays as given, host arrays copied
// into the context's staging buffer on stream s.
int ray_ptrs(vrc_ctx *c, const vrc_rays *r, cudaStream_t s, RayPtrs *out) {
  RayPtrs rp;
  rp.aos = nullptr;
  rp.n = r->n;
  if (r->on_device) {
    rp.x = r->x; rp.y = r->y; rp.z = r->z; rp.u = r->u;
    rp.v = r->v; rp.w = r->w; rp.E = r->E; rp.wt = r->wt;
  } else {
    const size_t bytes = sizeof(float) * (size_t)r->n;
    VRC_CUDA(c->stage.ensure(8 * bytes), "allocating ray staging");
    float *base = static_cast<float *>(c->stage.p);
    const float *src[8] = {r->x, r->y, r->z, r->u, r->v, r->w, r->E, r->wt};
    const float **dst[8] = {&rp.x, &rp.y, &rp.z, &rp.u, &rp.v, &rp.w, &rp.E, &rp.wt};
    for (int k = 0; k < 8; ++k) {
      float *dk = base + (size_t)k * r->n;
      VRC_CUDA(cudaMemcpyAsync(dk, src[k], bytes, cudaMemcpyHostToDevice, s), "copying rays to the device");
      *dst[k] = dk;
    }
  }
  *out = rp;
  return VRC_OK;
}

}  // namespace

// Host batches above this many rays are uploaded and cast chunk by chunk.
constexpr int64_t kUploadChunk = (int64_t)1 << 22;

// Cast of a large host batch with the upload overlapped: chunk i+1 is copied
// on the context's copy stream while chunk i is sorted and cast on stream s.
// Each chunk's cast waits for its upload (event), and an upload into a slot
// waits for the cast that last read that slot (event; this also orders a
// call after the previous call's casts).  Returns once every upload has
// completed, so the caller may reuse its host arrays.
int cast_host_pipelined(vrc_ctx *c, const vrc_rays *r, cudaStream_t s) {
  if (!c->up_stream) {
    VRC_CUDA(cudaStreamCreateWithFlags(&c->up_stream, cudaStreamNonBlocking), "creating the upload stream");
    for (int i = 0; i < 2; ++i) {
      VRC_CUDA(cudaEventCreateWithFlags(&c->up_copied[i], cudaEventDisableTiming), "creating an upload event");
      VRC_CUDA(cudaEventCreateWithFlags(&c->up_freed[i], cudaEventDisableTiming), "creating an upload event");
    }
  }
  const size_t slot_bytes = 8 * sizeof(float) * (size_t)kUploadChunk;
  for (int i = 0; i < 2; ++i) VRC_CUDA(c->up_slot[i].ensure(slot_bytes), "allocating upload slots");
  const float *src[8] = {r->x, r->y, r->z, r->u, r->v, r->w, r->E, r->wt};
  int last = 0;
  for (int64_t off = 0, i = 0; off < r->n; off += kUploadChunk, ++i) {
    const int slot = (int)(i & 1);
    const int64_t m = std::min(kUploadChunk, r->n - off);
    float *base = static_cast<float *>(c->up_slot[slot].p);
    VRC_CUDA(cudaStreamWaitEvent(c->up_stream, c->up_freed[slot], 0), "ordering an upload");
    RayPtrs rp;
    rp.aos = nullptr;
    rp.n = m;
    const float **dst[8] = {&rp.x, &rp.y, &rp.z, &rp.u, &rp.v, &rp.w, &rp.E, &rp.wt};
    for (int k = 0; k < 8; ++k) {
      float *dk = base + (size_t)k * m;
      VRC_CUDA(cudaMemcpyAsync(dk, src[k] + off, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, c->up_stream),
               "copying rays to the device");
      *dst[k] = dk;
    }
    VRC_CUDA(cudaEventRecord(c->up_copied[slot], c->up_stream), "recording an upload");
    VRC_CUDA(cudaStreamWaitEvent(s, c->up_copied[slot], 0), "ordering a cast after its upload");
    int rc = cast_device(c, rp, s);
    if (rc) return rc;
    VRC_CUDA(cudaEventRecord(c->up_freed[slot], s), "recording a cast");
    last = slot;
  }
  // uploads run in order on one stream: the last one done means all are
  VRC_CUDA(cudaEventSynchronize(c->up_copied[last]), "waiting for the ray upload");
  return VRC_OK;
}

extern "C" {

void vrc_default_options(vrc_options *opt) {
  if (!opt) return;
  opt->form = VRC_FORM_PLAIN;
  opt->sort = -1;
  opt->sort_len_buckets = -1;
  opt->block = 0;
  opt->blocks_per_sm = 0;
  opt->device = -1;
  opt->stop_at_zero = 0;
}

int vrc_create_mesh(const vrc_mesh_desc *d, const vrc_options *opt, vrc_ctx **out) {
  if (!out) return fail(VRC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(VRC_ERR_ARG, "mesh descriptor is NULL");
  if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0)
    return fail(VRC_ERR_ARG, "mesh dimensions must be positive (got %d x %d x %d)", d->nx, d->ny, d->nz);
  if ((int64_t)d->nx + d->ny + d->nz > (1 << 24))
    return fail(VRC_ERR_ARG, "mesh too large: nx+ny+nz must stay below 2^24");
  if (!finite_pos(d->dx) || !finite_pos(d->dy) || !finite_pos(d->dz))
    return fail(VRC_ERR_ARG, "cell spacings must be finite and positive");
  if (!std::isfinite(d->x0) || !std::isfinite(d->y0) || !std::isfinite(d->z0))
    return fail(VRC_ERR_ARG, "mesh origin must be finite");
  if (!d->material) return fail(VRC_ERR_ARG, "material array is NULL");
  if (d->n_materials < 1 || d->n_materials > kMaxMaterials)
    return fail(VRC_ERR_ARG, "n_materials must be in 1..%d", kMaxMaterials);
  if (d->n_groups < 1 || d->n_groups > kMaxGroups)
    return fail(VRC_ERR_ARG, "n_groups must be in 1..%d", kMaxGroups);
  if (!d->group_edges && d->n_groups != 1)
    return fail(VRC_ERR_ARG, "group_edges is NULL but n_groups is %d", d->n_groups);
  if (d->group_edges) {
    for (int g = 0; g <= d->n_groups; ++g) {
      if (!std::isfinite(d->group_edges[g]))
        return fail(VRC_ERR_ARG, "group edge %d is not finite", g);
      if (g > 0 && !(d->group_edges[g] > d->group_edges[g - 1]))
        return fail(VRC_ERR_ARG, "group edges must be strictly ascending");
    }
  }
  vrc_options o;
  vrc_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(&o);
  if (rc) return rc;

  const int64_t ncells = (int64_t)d->nx * d->ny * d->nz;
  std::vector<uint8_t> used(d->n_materials, 0);
  for (int64_t i = 0; i < ncells; ++i) {
    uint8_t m = d->material[i];
    if (m >= d->n_materials)
      return fail(VRC_ERR_ARG, "cell %lld has material %d >= n_materials %d", (long long)i, m, d->n_materials);
    used[m] = 1;
  }

  int dev = o.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess)
    return fail(VRC_ERR_CUDA, "no CUDA device available");
  DeviceGuard g(dev);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", dev);

  vrc_ctx *c = new (std::nothrow) vrc_ctx();
  if (!c) return fail(VRC_ERR_OOM, "out of host memory");
  c->device = dev;
  c->opt = o;
  c->n[0] = d->nx; c->n[1] = d->ny; c->n[2] = d->nz;
  c->org[0] = d->x0; c->org[1] = d->y0; c->org[2] = d->z0;
  c->h[0] = d->dx; c->h[1] = d->dy; c->h[2] = d->dz;
  c->ncells = ncells;
  c->n_materials = d->n_materials;
  c->n_groups = d->n_groups;
  if (d->group_edges) c->edges.assign(d->group_edges, d->group_edges + d->n_groups + 1);
  c->used = used;
  c->tabE.resize(d->n_materials);
  c->tabS.resize(d->n_materials);
  c->loaded.assign(d->n_materials, 0);

  auto bail = [&](int code) { delete c; return code; };
  cudaError_t e;
  if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return bail(cuda_fail(e, "querying the SM count"));
  if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(e, "creating the context stream"));
  const size_t tally_bytes = sizeof(double) * (size_t)ncells * d->n_groups;
  if ((e = cudaMalloc((void **)&c->d_mat, (size_t)ncells)) != cudaSuccess ||
      (e = cudaMalloc((void **)&c->d_tally, tally_bytes)) != cudaSuccess ||
      (e = cudaMalloc((void **)&c->d_counters, sizeof(unsigned long long) * kNumCounters)) != cudaSuccess ||
      (e = cudaMalloc((void **)&c->d_status, sizeof(unsigned))) != cudaSuccess)
    return bail(cuda_fail(e, "allocating the mesh and tally"));
  if (d->group_edges &&
      (e = cudaMalloc((void **)&c->d_edges, sizeof(double) * (d->n_groups + 1))) != cudaSuccess)
    return bail(cuda_fail(e, "allocating the group edges"));
  if ((e = cudaMemcpy(c->d_mat, d->material, (size_t)ncells, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(cuda_fail(e, "uploading the mesh"));
  if (d->group_edges &&
      (e = cudaMemcpy(c->d_edges, d->group_edges, sizeof(double) * (d->n_groups + 1),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(cuda_fail(e, "uploading the group edges"));
  if ((e = cudaMemsetAsync(c->d_tally, 0, tally_bytes, c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * kNumCounters, c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return bail(cuda_fail(e, "zeroing the tally"));
  *out = c;
  return VRC_OK;
}

int vrc_create_rect_mesh(const vrc_rect_mesh_desc *d, const vrc_options *opt, vrc_ctx **out) {
  if (!out) return fail(VRC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(VRC_ERR_ARG, "mesh descriptor is NULL");
  const int32_t n[3] = {d->nx, d->ny, d->nz};
  const double *e[3] = {d->x_edges, d->y_edges, d->z_edges};
  for (int k = 0; k < 3; ++k) {
    if (n[k] <= 0) return fail(VRC_ERR_ARG, "mesh dimensions must be positive (got %d x %d x %d)", d->nx, d->ny, d->nz);
    if (!e[k]) return fail(VRC_ERR_ARG, "edge array %d is NULL", k);
    for (int32_t j = 0; j <= n[k]; ++j) {
      if (!std::isfinite(e[k][j])) return fail(VRC_ERR_ARG, "edge %d of axis %d is not finite", j, k);
      if (j > 0 && !(e[k][j] > e[k][j - 1])) return fail(VRC_ERR_ARG, "edges of axis %d must be strictly ascending", k);
    }
  }
  vrc_mesh_desc u;
  u.nx = d->nx; u.ny = d->ny; u.nz = d->nz;
  u.x0 = e[0][0]; u.y0 = e[1][0]; u.z0 = e[2][0];
  u.dx = (e[0][n[0]] - e[0][0]) / n[0];
  u.dy = (e[1][n[1]] - e[1][0]) / n[1];
  u.dz = (e[2][n[2]] - e[2][0]) / n[2];
  u.material = d->material;
  u.n_materials = d->n_materials;
  u.n_groups = d->n_groups;
  u.group_edges = d->group_edges;
  vrc_ctx *c = nullptr;
  int rc = vrc_create_mesh(&u, opt, &c);
  if (rc) return rc;
  DeviceGuard g(c->device);
  const int64_t planes = (int64_t)n[0] + n[1] + n[2] + 3;
  std::vector<float2> df2(planes);
  std::vector<double> dd(planes), width(planes - 3);
  int64_t o = 0, ow = 0;
  for (int k = 0; k < 3; ++k) {
    c->rect_off[k] = o;
    for (int32_t j = 0; j <= n[k]; ++j, ++o) {
      const df sp = split(e[k][j]);
      df2[o] = make_float2(sp.hi, sp.lo);
      dd[o] = e[k][j];
      if (j < n[k]) width[ow++] = e[k][j + 1] - e[k][j];
    }
  }
  cudaError_t err;
  if ((err = c->rectDf.ensure(sizeof(float2) * planes)) != cudaSuccess ||
      (err = c->rectD.ensure(sizeof(double) * planes)) != cudaSuccess ||
      (err = c->rectWidth.ensure(sizeof(double) * width.size())) != cudaSuccess ||
      (err = cudaMemcpy(c->rectDf.p, df2.data(), sizeof(float2) * planes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(c->rectD.p, dd.data(), sizeof(double) * planes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(c->rectWidth.p, width.data(), sizeof(double) * width.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    delete c;
    return cuda_fail(err, "uploading the mesh planes");
  }
  c->rect = true;
  *out = c;
  return VRC_OK;
}

int vrc_load_xs(vrc_ctx *c, int32_t material, const double *E_eV, const double *sigma_t, int64_t n) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (material < 0 || material >= c->n_materials)
    return fail(VRC_ERR_ARG, "material %d out of range 0..%d", material, c->n_materials - 1);
  if (n < 0) return fail(VRC_ERR_ARG, "table length is negative");
  if (n > 0 && (!E_eV || !sigma_t)) return fail(VRC_ERR_ARG, "table arrays are NULL");
  if (n > ((int64_t)1 << 28)) return fail(VRC_ERR_ARG, "table too long");
  for (int64_t i = 0; i < n; ++i) {
    if (!finite_pos(E_eV[i])) return fail(VRC_ERR_ARG, "energy %lld is not finite and positive", (long long)i);
    if (i > 0 && !(E_eV[i] > E_eV[i - 1]))
      return fail(VRC_ERR_ARG, "energies must be strictly ascending (index %lld)", (long long)i);
    if (!std::isfinite(sigma_t[i]) || sigma_t[i] < 0.0)
      return fail(VRC_ERR_ARG, "sigma_t %lld is negative or not finite", (long long)i);
  }
  c->tabE[material].assign(E_eV, E_eV + n);
  c->tabS[material].assign(sigma_t, sigma_t + n);
  c->loaded[material] = 1;
  c->xs_dirty = true;
  return VRC_OK;
}

int vrc_cast_rays(vrc_ctx *c, const vrc_rays *r, void *cuda_stream) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (!r) return fail(VRC_ERR_ARG, "rays is NULL");
  if (r->n < 0) return fail(VRC_ERR_ARG, "ray count is negative");
  if (r->n == 0) return VRC_OK;
  if (!r->x || !r->y || !r->z || !r->u || !r->v || !r->w || !r->E || !r->wt)
    return fail(VRC_ERR_ARG, "a ray array is NULL");
  DeviceGuard g(c->device);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", c->device);
  if (c->xs_dirty) {
    int rc = build_xs(c);
    if (rc) {
      c->xs_dirty = true;
      return rc;
    }
  }
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  if (!r->on_device && r->n > kUploadChunk) return cast_host_pipelined(c, r, s);
  RayPtrs rp;
  {
    int rc = ray_ptrs(c, r, s, &rp);
    if (rc) return rc;
  }
  cudaEvent_t uploaded = nullptr;
  if (!r->on_device) {
    VRC_CUDA(c->get_event(&uploaded), "creating the upload event");
    VRC_CUDA(cudaEventRecord(uploaded, s), "recording the upload event");
  }
  {
    int rc = cast_device(c, rp, s);
    if (rc) return rc;
  }
  if (uploaded) {
    // the caller may reuse its host arrays once the copies have completed
    VRC_CUDA(cudaEventSynchronize(uploaded), "waiting for the ray upload");
    c->event_pool.push_back(uploaded);
  }
  return VRC_OK;
}

int vrc_sync(vrc_ctx *c, void *cuda_stream, vrc_stats *stats) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  DeviceGuard g(c->device);
  int rc = sync_streams(c, cuda_stream);
  if (rc) return rc;
  unsigned long long cnt[kNumCounters];
  unsigned st = 0;
  VRC_CUDA(cudaMemcpy(cnt, c->d_counters, sizeof cnt, cudaMemcpyDeviceToHost), "reading counters");
  VRC_CUDA(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost), "reading status");
  if (stats) {
    stats->segments = (int64_t)cnt[kCntSegments];
    stats->rays = (int64_t)cnt[kCntRays];
    stats->rejected = (int64_t)cnt[kCntRejected];
    stats->overflow = (int64_t)cnt[kCntOverflow];
  }
  return status_code(st);
}

int vrc_read_tally(vrc_ctx *c, double *out_host, int64_t n, int32_t flags, void *cuda_stream) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (!out_host) return fail(VRC_ERR_ARG, "output array is NULL");
  const int64_t total = c->ncells * c->n_groups;
  if (n != total) return fail(VRC_ERR_ARG, "tally has %lld entries, caller gave %lld", (long long)total, (long long)n);
  if (flags & ~VRC_PER_VOLUME) return fail(VRC_ERR_ARG, "unknown flags 0x%x", flags);
  DeviceGuard g(c->device);
  int rc = sync_streams(c, cuda_stream);
  if (rc) return rc;
  if (flags & VRC_PER_VOLUME) {
    const double scale = 1.0 / (c->h[0] * c->h[1] * c->h[2]);
    const int64_t chunk = std::min<int64_t>(total, (int64_t)8 << 20);
    VRC_CUDA(c->scratch.ensure(sizeof(double) * chunk), "allocating tally staging");
    for (int64_t off = 0; off < total; off += chunk) {
      const int64_t m = std::min(chunk, total - off);
      if (c->rect) {
        const double *w = static_cast<const double *>(c->rectWidth.p);
        VRC_CUDA(launch_per_volume_rect(c->d_tally + off, static_cast<double *>(c->scratch.p), m, off, c->n[0],
                                        c->n[1], c->ncells, w, w + c->n[0], w + c->n[0] + c->n[1], c->stream),
                 "launching the tally finalize kernel");
      } else {
        VRC_CUDA(launch_scale_copy(c->d_tally + off, static_cast<double *>(c->scratch.p), m, scale, c->stream),
                 "launching the tally finalize kernel");
      }
      VRC_CUDA(cudaMemcpyAsync(out_host + off, c->scratch.p, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream),
               "copying the tally");
      VRC_CUDA(cudaStreamSynchronize(c->stream), "copying the tally");
    }
  } else {
    VRC_CUDA(cudaMemcpyAsync(out_host, c->d_tally, sizeof(double) * total, cudaMemcpyDeviceToHost, c->stream),
             "copying the tally");
    VRC_CUDA(cudaStreamSynchronize(c->stream), "copying the tally");
  }
  unsigned st = 0;
  VRC_CUDA(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost), "reading status");
  return status_code(st);
}

double *vrc_tally_device_ptr(vrc_ctx *c) { return c ? c->d_tally : nullptr; }

void *vrc_context_stream(vrc_ctx *c) { return c ? static_cast<void *>(c->stream) : nullptr; }

int vrc_reset_tally(vrc_ctx *c, void *cuda_stream) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  DeviceGuard g(c->device);
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  VRC_CUDA(cudaMemsetAsync(c->d_tally, 0, sizeof(double) * c->ncells * c->n_groups, s), "zeroing the tally");
  VRC_CUDA(cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * kNumCounters, s), "zeroing counters");
  VRC_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s), "zeroing status");
  return VRC_OK;
}

int vrc_set_options(vrc_ctx *c, const vrc_options *opt) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (!opt) return fail(VRC_ERR_ARG, "options are NULL");
  int rc = check_options(opt);
  if (rc) return rc;
  int dev = c->device;
  c->opt = *opt;
  c->opt.device = dev;
  return VRC_OK;
}

void vrc_destroy(vrc_ctx *c) { delete c; }

const char *vrc_last_error(void) { return g_last_error.c_str(); }

int vrc_enable_timing(vrc_ctx *c, int32_t on) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  c->timing = on != 0;
  return VRC_OK;
}

int vrc_get_timing(vrc_ctx *c, void *cuda_stream, double *cast_ms, double *sort_ms,
                   int64_t *cast_launches, int32_t reset) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  DeviceGuard g(c->device);
  int rc = sync_streams(c, cuda_stream);
  if (rc) return rc;
  for (auto &t : c->pending) {
    float ms = 0.f;
    VRC_CUDA(cudaEventSynchronize(t.stop), "waiting for a timing event");
    VRC_CUDA(cudaEventElapsedTime(&ms, t.start, t.stop), "reading a timing event");
    (t.kind == 0 ? c->cast_ms : c->sort_ms) += ms;
    c->event_pool.push_back(t.start);
    c->event_pool.push_back(t.stop);
  }
  c->pending.clear();
  if (cast_ms) *cast_ms = c->cast_ms;
  if (sort_ms) *sort_ms = c->sort_ms;
  if (cast_launches) *cast_launches = c->cast_launches;
  if (reset) {
    c->cast_ms = c->sort_ms = 0.0;
    c->cast_launches = 0;
  }
  return VRC_OK;
}

int64_t vrc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"

// Internal accessors for vrc_static.cu (the no-allocation sort).
int vrc::set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }

int vrc::ctx_sort_args(const vrc_ctx *c, SortKeyArgs *P, const double **edges, int *device,
                       cudaStream_t *stream) {
  std::memset(P, 0, sizeof *P);
  for (int k = 0; k < 3; ++k) {
    P->lo[k] = (float)c->org[k];
    P->hi[k] = (float)(c->org[k] + c->n[k] * c->h[k]);
    P->inv_h[k] = (float)(1.0 / c->h[k]);
    P->n[k] = c->n[k];
  }
  P->n_groups = c->n_groups;
  int nl = c->opt.sort_len_buckets > 0 ? c->opt.sort_len_buckets : 64;
  while (nl > 1 && (int64_t)c->n_groups * nl + 1 > 16384) nl >>= 1;
  P->n_len = nl;
  const int max_cells = c->n[0] + c->n[1] + c->n[2] + 1;
  P->len_width = std::max(1, (max_cells + nl - 1) / nl);
  P->n_keys = c->n_groups * nl + 1;
  *edges = c->edges.empty() ? nullptr : c->d_edges;
  *device = c->device;
  *stream = c->stream;
  return VRC_OK;
}

extern "C" {

int vrc_device_count(void) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) return 0;
  return n;
}

int vrc_version(void) { return VRC_VERSION; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched form: a plan over many contexts, cast by one persistent kernel.
// ---------------------------------------------------------------------------
struct vrc_batch {
  int device = 0, form = 0;
  cudaStream_t stream = nullptr;
  vrc_batch_options opt;
  std::vector<vrc_ctx *> ctxs;
  int64_t total_rays = 0;
  CastArgs *d_probs = nullptr;
  BatchItem *d_items = nullptr;
  int n_items = 0;
  unsigned int *d_queue = nullptr;
  BatchShape shape{0, 0, 0};
  int grid = 0, block = 256;
  bool sorted = false;
  BSortProblem *d_bprobs = nullptr;
  int32_t *d_chunk_problem = nullptr;
  BSortPlan bplan;
  uint32_t *d_keys = nullptr, *d_table = nullptr, *d_offsets = nullptr, *d_tiles = nullptr;
  float *d_sorted = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels_per_launch = 0;

  ~vrc_batch() {
    DeviceGuard g(device);
    if (stream) cudaStreamSynchronize(stream);
    if (cap_stream) cudaStreamSynchronize(cap_stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cudaFree(d_probs);
    cudaFree(d_items);
    cudaFree(d_queue);
    cudaFree(d_bprobs);
    cudaFree(d_chunk_problem);
    cudaFree(d_keys);
    cudaFree(d_table);
    cudaFree(d_offsets);
    cudaFree(d_tiles);
    cudaFree(d_sorted);
  }
};

namespace {

int check_batch_options(const vrc_batch_options *o) {
  if (o->block < 0 || o->block > 256 || (o->block % 32) != 0)
    return fail(VRC_ERR_ARG, "batch block must be 0 or a multiple of 32 up to 256");
  if (o->blocks_per_sm < 0) return fail(VRC_ERR_ARG, "batch blocks_per_sm must be >= 0");
  if (o->chunk != 0 && (o->chunk < 64 || o->chunk > 65536))
    return fail(VRC_ERR_ARG, "batch chunk must be 0 or 64..65536");
  if (o->sort_len_buckets < -1 || o->sort_len_buckets > 256)
    return fail(VRC_ERR_ARG, "batch sort_len_buckets must be -1, 0 or 1..256");
  return VRC_OK;
}

// Enqueues the launch sequence of a plan on stream s.
cudaError_t enqueue_batch(vrc_batch *b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (b->sorted) {
    RayOut o;
    std::memset(&o, 0, sizeof o);
    o.aos = reinterpret_cast<float4 *>(b->d_sorted);  // sorted copy as 32-byte records
    e = launch_batched_sort(b->d_bprobs, b->d_chunk_problem, b->bplan, b->d_keys, b->d_table,
                            b->d_offsets, b->d_tiles, o, s);
    if (e != cudaSuccess) return e;
  }
  return launch_batched_cast(b->form, b->d_probs, b->d_items, b->n_items, b->d_queue, b->shape,
                             b->grid, b->block, s);
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(src.size(), 1));
  if (e != cudaSuccess) return e;
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

void vrc_default_batch_options(vrc_batch_options *opt) {
  if (!opt) return;
  opt->block = 0;
  opt->blocks_per_sm = 0;
  opt->chunk = 0;
  opt->sort_len_buckets = -1;
  opt->use_graph = 1;
}

int vrc_batch_create(vrc_ctx *const *ctxs, const vrc_rays *rays, int32_t n_problems,
                     const vrc_batch_options *opt, vrc_batch **out) {
  if (!out) return fail(VRC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || !rays || n_problems <= 0) return fail(VRC_ERR_ARG, "need at least one problem");
  vrc_batch_options o;
  vrc_default_batch_options(&o);
  if (opt) o = *opt;
  int rc = check_batch_options(&o);
  if (rc) return rc;
  const int dev = ctxs[0] ? ctxs[0]->device : -1;
  const int form = ctxs[0] ? ctxs[0]->opt.form : 0;
  int64_t total = 0;
  for (int p = 0; p < n_problems; ++p) {
    if (!ctxs[p]) return fail(VRC_ERR_ARG, "context %d is NULL", p);
    if (ctxs[p]->device != dev) return fail(VRC_ERR_ARG, "all contexts must be on one device");
    if (ctxs[p]->opt.form != form) return fail(VRC_ERR_ARG, "all contexts must use one precision form");
    const vrc_rays &r = rays[p];
    if (!r.on_device) return fail(VRC_ERR_ARG, "problem %d: the batched form takes device rays", p);
    if (ctxs[p]->rect) return fail(VRC_ERR_ARG, "problem %d: the batched form takes uniform meshes", p);
    if (r.n < 0) return fail(VRC_ERR_ARG, "problem %d: negative ray count", p);
    if (r.n > 0 && (!r.x || !r.y || !r.z || !r.u || !r.v || !r.w || !r.E || !r.wt))
      return fail(VRC_ERR_ARG, "problem %d: a ray array is NULL", p);
    total += r.n;
  }
  if (total >= ((int64_t)1 << 32)) return fail(VRC_ERR_ARG, "a batch holds fewer than 2^32 rays");
  DeviceGuard g(dev);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", dev);
  for (int p = 0; p < n_problems; ++p) {
    if (ctxs[p]->xs_dirty) {
      rc = build_xs(ctxs[p]);
      if (rc) {
        ctxs[p]->xs_dirty = true;
        return rc;
      }
    }
  }

  vrc_batch *b = new (std::nothrow) vrc_batch();
  if (!b) return fail(VRC_ERR_OOM, "out of host memory");
  auto bail = [&](int code) { delete b; return code; };
  b->device = dev;
  b->form = form;
  b->opt = o;
  b->stream = ctxs[0]->stream;
  b->ctxs.assign(ctxs, ctxs + n_problems);
  b->total_rays = total;
  const int chunk = o.chunk > 0 ? o.chunk : 2048;
  const int nl = o.sort_len_buckets < 0 ? 16 : o.sort_len_buckets;
  b->sorted = nl > 0 && total > 0;
  cudaError_t e;

  // order problems by decreasing walk length so the long ones start first
  std::vector<int> order(n_problems);
  for (int p = 0; p < n_problems; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const vrc_ctx *A = ctxs[a], *C = ctxs[c];
    return (A->n[0] + A->n[1] + A->n[2]) > (C->n[0] + C->n[1] + C->n[2]);
  });

  std::vector<int64_t> ray_base(n_problems, 0);
  {
    int64_t acc = 0;
    for (int p = 0; p < n_problems; ++p) { ray_base[p] = acc; acc += rays[p].n; }
  }
  if (b->sorted) {
    const size_t T = (size_t)total;
    std::vector<BSortProblem> bp(n_problems);
    std::vector<int32_t> chunk_problem;
    int64_t table = 0;
    int max_keys = 1;
    for (int p = 0; p < n_problems; ++p) {
      BSortProblem &q = bp[p];
      std::memset(&q, 0, sizeof q);
      const vrc_ctx *c = ctxs[p];
      for (int k = 0; k < 3; ++k) {
        q.P.lo[k] = (float)c->org[k];
        q.P.hi[k] = (float)(c->org[k] + c->n[k] * c->h[k]);
        q.P.inv_h[k] = (float)(1.0 / c->h[k]);
        q.P.n[k] = c->n[k];
      }
      q.P.n_groups = c->n_groups;
      int len = nl;
      while (len > 1 && (int64_t)c->n_groups * len + 1 > 16384) len >>= 1;
      q.P.n_len = len;
      q.P.len_width = std::max(1, (c->n[0] + c->n[1] + c->n[2] + 1 + len - 1) / len);
      q.P.n_keys = c->n_groups * len + 1;
      max_keys = std::max(max_keys, q.P.n_keys);
      q.edges = c->edges.empty() ? nullptr : c->d_edges;
      const vrc_rays &r = rays[p];
      q.src.x = r.x; q.src.y = r.y; q.src.z = r.z; q.src.u = r.u;
      q.src.v = r.v; q.src.w = r.w; q.src.E = r.E; q.src.wt = r.wt;
      q.src.n = r.n;
      q.ray_base = ray_base[p];
      q.n_chunks = (int32_t)((r.n + b->bplan.chunk - 1) / b->bplan.chunk);
      q.first_chunk = (int32_t)chunk_problem.size();
      q.table_base = table;
      table += (int64_t)q.P.n_keys * q.n_chunks;
      for (int c2 = 0; c2 < q.n_chunks; ++c2) chunk_problem.push_back(p);
    }
    b->bplan.n_chunks = (int)chunk_problem.size();
    b->bplan.table_len = table;
    b->bplan.n_tiles = (int)((table + scan_tile_elems() - 1) / scan_tile_elems());
    b->bplan.max_keys = max_keys;
    b->bplan.total_rays = total;
    if ((e = upload(&b->d_bprobs, bp)) != cudaSuccess || (e = upload(&b->d_chunk_problem, chunk_problem)) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_keys, sizeof(uint32_t) * T)) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_table, sizeof(uint32_t) * std::max<int64_t>(table, 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_offsets, sizeof(uint32_t) * std::max<int64_t>(table, 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_tiles, sizeof(uint32_t) * std::max(b->bplan.n_tiles, 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_sorted, 8 * sizeof(float) * T)) != cudaSuccess)
      return bail(cuda_fail(e, "allocating the batch sort"));
    if ((e = prepare_batched_sort(b->bplan)) != cudaSuccess) return bail(cuda_fail(e, "preparing the batch sort"));
  }

  std::vector<CastArgs> probs(n_problems);
  BatchShape sh{0, 0, 0};
  for (int p = 0; p < n_problems; ++p) {
    RayPtrs rp;
    std::memset(&rp, 0, sizeof rp);
    if (b->sorted) {
      rp.aos = reinterpret_cast<const float4 *>(b->d_sorted);
      rp.n = total;
    } else {
      const vrc_rays &r = rays[p];
      rp.x = r.x; rp.y = r.y; rp.z = r.z; rp.u = r.u; rp.v = r.v; rp.w = r.w; rp.E = r.E; rp.wt = r.wt;
      rp.n = r.n;
    }
    probs[p] = make_args(ctxs[p], rp);
    sh.max_hash = std::max(sh.max_hash, ctxs[p]->n_union > 0 ? ctxs[p]->n_hash : 0);
    sh.max_groups = std::max(sh.max_groups, ctxs[p]->n_groups);
    sh.max_mat = std::max(sh.max_mat, ctxs[p]->n_materials);
  }
  b->shape = sh;
  std::vector<BatchItem> items;
  for (int q = 0; q < n_problems; ++q) {
    const int p = order[q];
    const int64_t n = rays[p].n;
    const int64_t base = b->sorted ? ray_base[p] : 0;
    for (int64_t s = 0; s < n; s += chunk) {
      BatchItem it;
      it.problem = p;
      it.start = base + s;
      it.count = (int32_t)std::min<int64_t>(chunk, n - s);
      items.push_back(it);
    }
  }
  if (items.size() >= ((size_t)1 << 31)) return bail(fail(VRC_ERR_ARG, "too many work items"));
  b->n_items = (int)items.size();
  if ((e = upload(&b->d_probs, probs)) != cudaSuccess || (e = upload(&b->d_items, items)) != cudaSuccess ||
      (e = cudaMalloc((void **)&b->d_queue, sizeof(unsigned int))) != cudaSuccess)
    return bail(cuda_fail(e, "allocating the batch plan"));

  b->block = o.block > 0 ? o.block : 256;
  int bps = o.blocks_per_sm;
  if ((e = batched_occupancy(form, sh, b->block, &bps)) != cudaSuccess)
    return bail(cuda_fail(e, "querying batch occupancy"));
  if (o.blocks_per_sm > 0) bps = std::min(bps, o.blocks_per_sm);
  if (bps <= 0) return bail(fail(VRC_ERR_ARG, "the batched kernel does not fit on an SM"));
  int sms = ctxs[0]->num_sms;
  b->grid = (int)std::min<int64_t>((int64_t)sms * bps, std::max(b->n_items, 1));

  if (o.use_graph) {
    if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(cuda_fail(e, "creating the capture stream"));
    const long long before = g_launches.load();
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return bail(cuda_fail(e, "beginning graph capture"));
    cudaError_t ee = enqueue_batch(b, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    b->kernels_per_launch = g_launches.load() - before;
    g_launches.fetch_sub(b->kernels_per_launch);
    if (ee != cudaSuccess) return bail(cuda_fail(ee, "capturing the batch"));
    if (e != cudaSuccess) return bail(cuda_fail(e, "ending graph capture"));
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
      return bail(cuda_fail(e, "instantiating the batch graph"));
  }
  *out = b;
  return VRC_OK;
}

int vrc_batch_launch(vrc_batch *b, void *cuda_stream) {
  if (!b) return fail(VRC_ERR_ARG, "batch is NULL");
  DeviceGuard g(b->device);
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : b->stream;
  if (b->exec) {
    VRC_CUDA(cudaGraphLaunch(b->exec, s), "launching the batch graph");
    g_launches.fetch_add(b->kernels_per_launch);
  } else {
    VRC_CUDA(enqueue_batch(b, s), "launching the batch");
  }
  return VRC_OK;
}

void vrc_batch_destroy(vrc_batch *b) { delete b; }

int vrc_cast_batched(vrc_ctx *const *ctxs, const vrc_rays *rays, int32_t n_problems, void *cuda_stream) {
  vrc_batch *b = nullptr;
  int rc = vrc_batch_create(ctxs, rays, n_problems, nullptr, &b);
  if (rc) return rc;
  rc = vrc_batch_launch(b, cuda_stream);
  if (rc == VRC_OK) {
    DeviceGuard g(b->device);
    cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : b->stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "waiting for the batch");
  }
  vrc_batch_destroy(b);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned cross-section surrogate.
// ---------------------------------------------------------------------------
namespace {

// lin-lin sigma of one material's own table at e (clamped), float64.
double table_sigma(const std::vector<double> &E, const std::vector<double> &S, double e) {
  const size_t n = E.size();
  if (n == 0) return 0.0;
  if (n == 1 || e <= E[0]) return S[0];
  if (e >= E[n - 1]) return S[n - 1];
  size_t k = std::upper_bound(E.begin(), E.end(), e) - E.begin() - 1;
  return S[k] + (e - E[k]) * (S[k + 1] - S[k]) / (E[k + 1] - E[k]);
}

uint64_t host_mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

struct TmpDev {  // device buffers freed at scope exit
  std::vector<void *> ptrs;
  cudaError_t alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~TmpDev() {
    for (void *p : ptrs) cudaFree(p);
  }
};

}  // namespace

extern "C" {

int vrc_mlp_forward(const float *params, const float *E, int64_t n, double e_lo, double e_hi,
                    float *log_sigma, void *cuda_stream) {
  if (!params || !E || !log_sigma || n < 0) return fail(VRC_ERR_ARG, "vrc_mlp_forward: bad arguments");
  if (!(e_lo > 0.0) || !(e_hi > e_lo)) return fail(VRC_ERR_ARG, "vrc_mlp_forward: need 0 < e_lo < e_hi");
  int dev = 0, sms = 0;
  VRC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  VRC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "querying the SM count");
  mlp::ApplyArgs a;
  std::memset(&a, 0, sizeof a);
  a.params = params;
  a.E = E;
  a.n = n;
  a.out = log_sigma;
  a.mode = 0;
  a.mat_mask = 0xffffu;
  a.emb = mlp::make_embed(e_lo, e_hi);
  VRC_CUDA(mlp::launch_apply(a, sms, static_cast<cudaStream_t>(cuda_stream)), "launching the surrogate forward");
  return VRC_OK;
}

int vrc_mlp_loss_grad(const float *params, const float *E, const float *target, const uint8_t *mask,
                      int64_t n, int64_t count, double e_lo, double e_hi, float *grad, float *loss,
                      void *cuda_stream) {
  if (!params || !E || !target || !grad || !loss || n < 0 || count <= 0)
    return fail(VRC_ERR_ARG, "vrc_mlp_loss_grad: bad arguments");
  if (!(e_lo > 0.0) || !(e_hi > e_lo)) return fail(VRC_ERR_ARG, "vrc_mlp_loss_grad: need 0 < e_lo < e_hi");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  VRC_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * mlp::kParams, s), "zeroing the gradient");
  VRC_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s), "zeroing the loss");
  mlp::TrainArgs a;
  std::memset(&a, 0, sizeof a);
  a.params = params;
  a.E = E;
  a.target = target;
  a.mask = mask;
  a.mat_mask = 0xffffu;
  a.m = n;
  a.inv_count = (float)(1.0 / (double)count);
  a.grad = grad;
  a.loss = loss;
  a.emb = mlp::make_embed(e_lo, e_hi);
  VRC_CUDA(mlp::launch_train(a, s), "launching the surrogate gradient");
  return VRC_OK;
}

void vrc_default_surrogate_options(vrc_surrogate_options *opt) {
  if (!opt) return;
  opt->steps = 8000;
  opt->batch = 4096;
  opt->lr = 5e-3f;
  opt->tol = 1e-3f;
  opt->seed = 4;
}

int vrc_train_surrogate(vrc_ctx *c, const vrc_surrogate_options *opt, vrc_surrogate_report *report) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  vrc_surrogate_options o;
  vrc_default_surrogate_options(&o);
  if (opt) o = *opt;
  if (o.steps < 0 || o.batch < 64 || o.batch > (1 << 22) || !(o.lr > 0.f) || !(o.tol > 0.f))
    return fail(VRC_ERR_ARG, "bad surrogate options");
  if (c->n_materials > mlp::kOut)
    return fail(VRC_ERR_ARG, "the surrogate models at most %d materials", mlp::kOut);
  DeviceGuard g(c->device);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", c->device);
  if (c->xs_dirty) {
    int rc = build_xs(c);
    if (rc) { c->xs_dirty = true; return rc; }
  }
  uint32_t mask = 0;
  for (int m = 0; m < c->n_materials; ++m)
    if (c->loaded[m] && !c->tabE[m].empty()) mask |= 1u << m;
  if (mask == 0 || c->n_union < 2) return fail(VRC_ERR_STATE, "no cross-section tables to learn");

  // energies: the union grid, refined; training at fractions 0, 1/4, 1/2,
  // 3/4 of every interval (plus the last point), validation at (k + 1/2)/8
  std::vector<double> U((size_t)c->n_union);
  VRC_CUDA(cudaMemcpy(U.data(), c->xsE.p, sizeof(double) * U.size(), cudaMemcpyDeviceToHost), "reading the grid");
  const int nm = c->n_materials;
  std::vector<float> trE, trT, vaE;
  std::vector<double> vaE64;
  for (size_t i = 0; i + 1 < U.size(); ++i) {
    for (int q = 0; q < 4; ++q) trE.push_back((float)(U[i] + (U[i + 1] - U[i]) * q / 4.0));
    for (int q = 0; q < 8; ++q) {
      const double e = U[i] + (U[i + 1] - U[i]) * (q + 0.5) / 8.0;
      vaE.push_back((float)e);
      vaE64.push_back((double)(float)e);
    }
  }
  trE.push_back((float)U.back());
  const int64_t n_tr = (int64_t)trE.size(), n_va = (int64_t)vaE.size();
  trT.assign((size_t)n_tr * mlp::kOut, 0.f);
  for (int64_t i = 0; i < n_tr; ++i)
    for (int m = 0; m < nm; ++m)
      if ((mask >> m) & 1u) {
        const double sg = table_sigma(c->tabE[m], c->tabS[m], (double)trE[i]);
        trT[(size_t)i * mlp::kOut + m] = (float)std::log(std::max(sg, 1e-300));
      }
  // a material whose table has a zero sigma is not modelled
  for (int m = 0; m < nm; ++m)
    if ((mask >> m) & 1u)
      for (double v : c->tabS[m])
        if (!(v > 0.0)) { mask &= ~(1u << m); break; }

  // initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases
  std::vector<float> P(mlp::kParams, 0.f);
  auto fill = [&](int off, int rows, int cols, uint64_t salt) {
    const float bound = 1.f / std::sqrt((float)cols);
    for (int i = 0; i < rows * cols; ++i) {
      const double u = (host_mix64(o.seed * 0x100000001B3ull + salt * 0x9E3779B9ull + i) >> 11) * (1.0 / 9007199254740992.0);
      P[off + i] = (float)((2.0 * u - 1.0) * bound);
    }
  };
  fill(mlp::kOffW1, mlp::kHid, mlp::kEmb, 1);
  fill(mlp::kOffW2, mlp::kHid, mlp::kHid, 2);
  fill(mlp::kOffW3, mlp::kOut, mlp::kHid, 3);

  TmpDev tmp;
  float *d_trE, *d_trT, *d_grad, *d_m1, *d_m2, *d_loss, *d_vaE, *d_vaY;
  VRC_CUDA(tmp.alloc((void **)&d_trE, sizeof(float) * n_tr), "allocating training data");
  VRC_CUDA(tmp.alloc((void **)&d_trT, sizeof(float) * trT.size()), "allocating training data");
  VRC_CUDA(tmp.alloc((void **)&d_grad, sizeof(float) * mlp::kParams), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_m1, sizeof(float) * mlp::kParams), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_m2, sizeof(float) * mlp::kParams), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_loss, sizeof(float) * (o.steps + 1)), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_vaE, sizeof(float) * n_va), "allocating validation data");
  VRC_CUDA(tmp.alloc((void **)&d_vaY, sizeof(float) * n_va * mlp::kOut), "allocating validation data");
  if (!(o.steps == 0 && c->mlp_ready))
    VRC_CUDA(c->mlpParams.ensure(sizeof(float) * mlp::kParams), "allocating the surrogate");
  VRC_CUDA(c->mlpFlags.ensure((size_t)c->n_hash), "allocating the surrogate flags");
  float *d_P = static_cast<float *>(c->mlpParams.p);
  cudaStream_t s = c->stream;
  VRC_CUDA(cudaMemcpy(d_trE, trE.data(), sizeof(float) * n_tr, cudaMemcpyHostToDevice), "uploading training data");
  VRC_CUDA(cudaMemcpy(d_trT, trT.data(), sizeof(float) * trT.size(), cudaMemcpyHostToDevice), "uploading training data");
  VRC_CUDA(cudaMemcpy(d_vaE, vaE.data(), sizeof(float) * n_va, cudaMemcpyHostToDevice), "uploading validation data");
  const bool revalidate = o.steps == 0;
  if (revalidate && !c->mlp_ready) return fail(VRC_ERR_STATE, "no trained surrogate to re-validate");
  if (!revalidate)
    VRC_CUDA(cudaMemcpy(d_P, P.data(), sizeof(float) * mlp::kParams, cudaMemcpyHostToDevice), "uploading weights");
  VRC_CUDA(cudaMemsetAsync(d_m1, 0, sizeof(float) * mlp::kParams, s), "zeroing Adam state");
  VRC_CUDA(cudaMemsetAsync(d_m2, 0, sizeof(float) * mlp::kParams, s), "zeroing Adam state");
  VRC_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float) * (o.steps + 1), s), "zeroing losses");

  const int n_out = __builtin_popcount(mask);
  mlp::TrainArgs ta;
  std::memset(&ta, 0, sizeof ta);
  ta.params = d_P;
  ta.E = d_trE;
  ta.target = d_trT;
  ta.mat_mask = mask;
  ta.m = o.batch;
  ta.set_n = n_tr;
  ta.inv_count = 1.f / (float)((int64_t)o.batch * n_out);
  ta.grad = d_grad;
  ta.emb = mlp::make_embed(U.front(), U.back());
  const int warm = std::min(200, std::max(1, o.steps / 20));
  for (int step = 1; step <= o.steps; ++step) {
    VRC_CUDA(cudaMemsetAsync(d_grad, 0, sizeof(float) * mlp::kParams, s), "zeroing the gradient");
    ta.seed = host_mix64(o.seed ^ ((uint64_t)step << 32));
    ta.loss = d_loss + step;
    VRC_CUDA(mlp::launch_train(ta, s), "launching a training step");
    const double prog = (double)(step - 1) / std::max(1, o.steps - 1);
    double lr = o.lr * (0.02 + 0.98 * 0.5 * (1.0 + std::cos(M_PI * prog)));
    if (step <= warm) lr *= (double)step / warm;
    VRC_CUDA(mlp::launch_adam(d_P, d_grad, d_m1, d_m2, mlp::kParams, (float)lr, 0.9f, 0.999f, 1e-8f, step, s),
             "launching Adam");
  }
  // validation
  mlp::ApplyArgs aa;
  std::memset(&aa, 0, sizeof aa);
  aa.params = d_P;
  aa.E = d_vaE;
  aa.n = n_va;
  aa.out = d_vaY;
  aa.mode = 0;
  aa.mat_mask = mask;
  aa.emb = ta.emb;
  aa.status = c->d_status;
  VRC_CUDA(mlp::launch_apply(aa, c->num_sms, s), "launching the validation pass");
  std::vector<float> Y((size_t)n_va * mlp::kOut), L((size_t)o.steps + 1, 0.f);
  VRC_CUDA(cudaStreamSynchronize(s), "training the surrogate");
  VRC_CUDA(cudaMemcpy(Y.data(), d_vaY, sizeof(float) * Y.size(), cudaMemcpyDeviceToHost), "reading validation");
  VRC_CUDA(cudaMemcpy(L.data(), d_loss, sizeof(float) * L.size(), cudaMemcpyDeviceToHost), "reading losses");

  std::vector<float> bin_err((size_t)c->n_hash, 0.f), all_err;
  all_err.reserve((size_t)n_va);
  const double l2a = std::log2(U.front());
  for (int64_t i = 0; i < n_va; ++i) {
    float worst = 0.f;
    for (int m = 0; m < nm; ++m) {
      if (!((mask >> m) & 1u)) continue;
      const double sg = table_sigma(c->tabE[m], c->tabS[m], vaE64[i]);
      const double got = std::exp((double)Y[(size_t)i * mlp::kOut + m]);
      worst = std::max(worst, (float)(std::fabs(got - sg) / sg));
    }
    int b = (int)std::floor((std::log2(vaE64[i]) - l2a) * c->inv_bw);
    b = std::min(std::max(b, 0), c->n_hash - 1);
    bin_err[b] = std::max(bin_err[b], worst);
    all_err.push_back(worst);
  }
  std::vector<uint8_t> flags((size_t)c->n_hash, 0);
  int accepted = 0;
  float max_acc = 0.f;
  for (int b = 0; b < c->n_hash; ++b) {
    bool bad = bin_err[b] > o.tol || !std::isfinite(bin_err[b]);
    if (b > 0) bad = bad || bin_err[b - 1] > o.tol;
    if (b + 1 < c->n_hash) bad = bad || bin_err[b + 1] > o.tol;
    flags[b] = bad ? 1 : 0;
    if (!bad) { ++accepted; max_acc = std::max(max_acc, bin_err[b]); }
  }
  VRC_CUDA(cudaMemcpy(c->mlpFlags.p, flags.data(), flags.size(), cudaMemcpyHostToDevice), "uploading flags");
  c->mlp_ready = true;
  c->mlp_mask = mask;
  c->mlp_lo = U.front();
  c->mlp_hi = U.back();
  if (report) {
    std::nth_element(all_err.begin(), all_err.begin() + all_err.size() / 2, all_err.end());
    report->final_loss = L.back();
    report->bins = c->n_hash;
    report->bins_accepted = accepted;
    report->coverage = (float)accepted / (float)c->n_hash;
    report->max_rel_err_accepted = max_acc;
    report->median_rel_err = all_err.empty() ? 0.f : all_err[all_err.size() / 2];
    report->train_points = n_tr;
    report->validation_points = n_va;
  }
  return VRC_OK;
}

int vrc_set_xs_mode(vrc_ctx *c, int32_t mode) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (mode != VRC_XS_TABLE && mode != VRC_XS_SURROGATE) return fail(VRC_ERR_ARG, "unknown lookup mode %d", mode);
  if (mode == VRC_XS_SURROGATE && !c->mlp_ready) return fail(VRC_ERR_STATE, "no surrogate has been trained");
  c->xs_mode = mode;
  return VRC_OK;
}

int vrc_get_surrogate_params(vrc_ctx *c, float *params_host) {
  if (!c || !params_host) return fail(VRC_ERR_ARG, "bad arguments");
  if (!c->mlp_ready) return fail(VRC_ERR_STATE, "no surrogate has been trained");
  DeviceGuard g(c->device);
  VRC_CUDA(cudaStreamSynchronize(c->stream), "synchronizing");
  VRC_CUDA(cudaMemcpy(params_host, c->mlpParams.p, sizeof(float) * mlp::kParams, cudaMemcpyDeviceToHost),
           "reading the surrogate");
  return VRC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Streaming ray buffers: fill / copy / cast overlapped across buffers.
// ---------------------------------------------------------------------------
struct vrc_stream {
  vrc_ctx *ctx = nullptr;
  int64_t capacity = 0;
  int n = 0;
  int cur = 0;          // buffer handed out by the next acquire
  bool held = false;    // an acquired buffer awaits submit
  cudaStream_t copy = nullptr;
  std::vector<vrc_ray_record *> host;
  std::vector<void *> dev;
  std::vector<cudaEvent_t> copied, cast;  // per buffer
  std::vector<bool> used;

  ~vrc_stream() {
    DeviceGuard g(ctx ? ctx->device : -1);
    if (copy) cudaStreamSynchronize(copy);
    if (ctx && ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto e : copied) if (e) cudaEventDestroy(e);
    for (auto e : cast) if (e) cudaEventDestroy(e);
    for (auto p : host) if (p) cudaFreeHost(p);
    for (auto p : dev) if (p) cudaFree(p);
    if (copy) cudaStreamDestroy(copy);
  }
};

extern "C" {

int vrc_stream_create(vrc_ctx *c, int64_t capacity, int32_t n_buffers, vrc_stream **out) {
  if (!out) return fail(VRC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (capacity <= 0 || capacity > ((int64_t)1 << 31)) return fail(VRC_ERR_ARG, "capacity must be in 1..2^31");
  if (n_buffers < 2 || n_buffers > 16) return fail(VRC_ERR_ARG, "n_buffers must be in 2..16");
  DeviceGuard g(c->device);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", c->device);
  vrc_stream *st = new (std::nothrow) vrc_stream();
  if (!st) return fail(VRC_ERR_OOM, "out of host memory");
  st->ctx = c;
  st->capacity = capacity;
  st->n = n_buffers;
  st->host.assign(n_buffers, nullptr);
  st->dev.assign(n_buffers, nullptr);
  st->copied.assign(n_buffers, nullptr);
  st->cast.assign(n_buffers, nullptr);
  st->used.assign(n_buffers, false);
  const size_t bytes = sizeof(vrc_ray_record) * (size_t)capacity;
  cudaError_t e;
  auto bail = [&](cudaError_t err, const char *what) { delete st; return cuda_fail(err, what); };
  if ((e = cudaStreamCreateWithFlags(&st->copy, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "creating the copy stream");
  for (int i = 0; i < n_buffers; ++i) {
    if ((e = cudaHostAlloc((void **)&st->host[i], bytes, cudaHostAllocDefault)) != cudaSuccess)
      return bail(e, "allocating a pinned ray buffer");
    if ((e = cudaMalloc(&st->dev[i], bytes)) != cudaSuccess) return bail(e, "allocating a device ray buffer");
    if ((e = cudaEventCreateWithFlags(&st->copied[i], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&st->cast[i], cudaEventDisableTiming)) != cudaSuccess)
      return bail(e, "creating stream events");
  }
  *out = st;
  return VRC_OK;
}

int vrc_stream_acquire(vrc_stream *s, vrc_ray_record **buffer, int64_t *capacity) {
  if (!s || !buffer) return fail(VRC_ERR_ARG, "bad arguments");
  DeviceGuard g(s->ctx->device);
  const int i = s->cur;
  if (!s->held && s->used[i])  // the host buffer is free once its last upload is done
    VRC_CUDA(cudaEventSynchronize(s->copied[i]), "waiting for a buffer's upload");
  s->held = true;
  *buffer = s->host[i];
  if (capacity) *capacity = s->capacity;
  return VRC_OK;
}

int vrc_stream_submit(vrc_stream *s, int64_t n) {
  if (!s) return fail(VRC_ERR_ARG, "stream is NULL");
  if (!s->held) return fail(VRC_ERR_STATE, "submit without an acquired buffer");
  if (n < 0 || n > s->capacity) return fail(VRC_ERR_ARG, "record count out of range");
  vrc_ctx *c = s->ctx;
  DeviceGuard g(c->device);
  const int i = s->cur;
  s->held = false;
  s->cur = (i + 1) % s->n;
  if (n == 0) return VRC_OK;
  if (c->xs_dirty) {
    int rc = build_xs(c);
    if (rc) { c->xs_dirty = true; return rc; }
  }
  // the device buffer is free once the cast that read it last has finished
  if (s->used[i]) VRC_CUDA(cudaStreamWaitEvent(s->copy, s->cast[i], 0), "ordering the upload");
  VRC_CUDA(cudaMemcpyAsync(s->dev[i], s->host[i], sizeof(vrc_ray_record) * (size_t)n,
                           cudaMemcpyHostToDevice, s->copy), "uploading a ray buffer");
  VRC_CUDA(cudaEventRecord(s->copied[i], s->copy), "recording the upload");
  VRC_CUDA(cudaStreamWaitEvent(c->stream, s->copied[i], 0), "ordering the cast");
  RayPtrs rp;
  std::memset(&rp, 0, sizeof rp);
  rp.aos = static_cast<const float4 *>(s->dev[i]);
  rp.n = n;
  int rc = cast_device(c, rp, c->stream);
  if (rc) return rc;
  VRC_CUDA(cudaEventRecord(s->cast[i], c->stream), "recording the cast");
  s->used[i] = true;
  return VRC_OK;
}

int vrc_stream_finish(vrc_stream *s) {
  if (!s) return fail(VRC_ERR_ARG, "stream is NULL");
  DeviceGuard g(s->ctx->device);
  VRC_CUDA(cudaStreamSynchronize(s->copy), "waiting for uploads");
  VRC_CUDA(cudaStreamSynchronize(s->ctx->stream), "waiting for casts");
  return VRC_OK;
}

void vrc_stream_destroy(vrc_stream *s) { delete s; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch moments of the tally.
// ---------------------------------------------------------------------------
extern "C" {

int vrc_moments_enable(vrc_ctx *c, int32_t mode) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (mode != VRC_MOMENTS_OFF && mode != VRC_MOMENTS_BATCH && mode != VRC_MOMENTS_HISTORY)
    return fail(VRC_ERR_ARG, "unknown moments mode %d", mode);
  DeviceGuard g(c->device);
  VRC_CUDA(cudaStreamSynchronize(c->stream), "synchronizing");
  c->batches = 0;
  c->moment_mode = mode;
  if (mode == VRC_MOMENTS_OFF) {
    c->momS1.release();
    c->momS2.release();
    c->histTab.release();
    c->histBits.release();
    c->histCap = 0;
    c->moments = false;
    return VRC_OK;
  }
  const size_t bytes = sizeof(double) * (size_t)(c->ncells * c->n_groups);
  VRC_CUDA(c->momS1.ensure(bytes), "allocating tally moments");
  VRC_CUDA(c->momS2.ensure(bytes), "allocating tally moments");
  VRC_CUDA(cudaMemsetAsync(c->momS1.p, 0, bytes, c->stream), "zeroing tally moments");
  VRC_CUDA(cudaMemsetAsync(c->momS2.p, 0, bytes, c->stream), "zeroing tally moments");
  c->moments = true;
  return VRC_OK;
}

int vrc_moments_fold(vrc_ctx *c, void *cuda_stream) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (!c->moments) return fail(VRC_ERR_STATE, "moments are not enabled");
  if (c->moment_mode != VRC_MOMENTS_BATCH) return fail(VRC_ERR_STATE, "moments are per history, not per batch");
  DeviceGuard g(c->device);
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  VRC_CUDA(launch_fold_moments(c->d_tally, static_cast<double *>(c->momS1.p),
                               static_cast<double *>(c->momS2.p), c->ncells * c->n_groups, s),
           "launching the moment fold");
  c->batches += 1;
  return VRC_OK;
}

int vrc_cast_histories(vrc_ctx *c, const vrc_rays *r, const uint32_t *history, int64_t n_histories,
                       void *cuda_stream) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (!r) return fail(VRC_ERR_ARG, "rays is NULL");
  if (r->n < 0 || n_histories < 0) return fail(VRC_ERR_ARG, "negative ray or history count");
  if (!c->moments || c->moment_mode != VRC_MOMENTS_HISTORY)
    return fail(VRC_ERR_STATE, "per-history moments are not enabled");
  if (c->ncells * c->n_groups >= (int64_t)0xffffffff)
    return fail(VRC_ERR_ARG, "per-history moments need fewer than 2^32 - 1 (group, cell) bins");
  if (r->n > 0 && (!history || !r->x || !r->y || !r->z || !r->u || !r->v || !r->w || !r->E || !r->wt))
    return fail(VRC_ERR_ARG, "a ray or history array is NULL");
  if (r->n == 0) {
    c->batches += n_histories;
    return VRC_OK;
  }
  DeviceGuard g(c->device);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", c->device);
  if (c->xs_dirty) {
    int rc = build_xs(c);
    if (rc) {
      c->xs_dirty = true;
      return rc;
    }
  }
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  RayPtrs rp;
  {
    int rc = ray_ptrs(c, r, s, &rp);
    if (rc) return rc;
  }
  const uint32_t *hist = history;
  if (!r->on_device) {
    VRC_CUDA(c->histIds.ensure(sizeof(uint32_t) * (size_t)r->n), "allocating history staging");
    VRC_CUDA(cudaMemcpyAsync(c->histIds.p, history, sizeof(uint32_t) * (size_t)r->n, cudaMemcpyHostToDevice, s),
             "copying history ids to the device");
    hist = static_cast<const uint32_t *>(c->histIds.p);
  }
  // table size: twice an upper bound of the call's segments, a power of two
  BoundGeom G;
  for (int k = 0; k < 3; ++k) {
    G.lo[k] = c->org[k];
    G.h[k] = c->h[k];
    G.n[k] = c->n[k];
    G.e[k] = c->rect ? static_cast<const double *>(c->rectD.p) + c->rect_off[k] : nullptr;
  }
  VRC_CUDA(c->histBound.ensure(sizeof(unsigned long long)), "allocating the segment bound");
  unsigned long long *d_bound = static_cast<unsigned long long *>(c->histBound.p);
  VRC_CUDA(cudaMemsetAsync(d_bound, 0, sizeof(unsigned long long), s), "zeroing the segment bound");
  VRC_CUDA(launch_segment_bound(G, rp, d_bound, c->num_sms, s), "launching the segment bound");
  unsigned long long bound = 0;
  VRC_CUDA(cudaMemcpyAsync(&bound, d_bound, sizeof bound, cudaMemcpyDeviceToHost, s), "reading the segment bound");
  VRC_CUDA(cudaStreamSynchronize(s), "waiting for the segment bound");  // host arrays are free from here
  unsigned long long cap = 1024;
  while (cap < 2 * bound) cap <<= 1;
  if (cap > c->histCap) {
    c->histTab.release();
    c->histBits.release();
    c->histCap = 0;
    size_t free_b = 0, total_b = 0;
    VRC_CUDA(cudaMemGetInfo(&free_b, &total_b), "querying device memory");
    const unsigned long long bytes = 16ull * cap + cap / 8ull;
    if (bytes > free_b / 10 * 9)
      return fail(VRC_ERR_OOM, "this call's histories need a %.1f GB table (%.1f GB free); split the call",
                  bytes / 1e9, free_b / 1e9);
    VRC_CUDA(c->histTab.ensure(16ull * cap), "allocating the per-history table");
    VRC_CUDA(c->histBits.ensure(cap / 8ull), "allocating the per-history table");
    VRC_CUDA(cudaMemsetAsync(c->histTab.p, 0, 16ull * cap, s), "clearing the per-history table");
    VRC_CUDA(cudaMemsetAsync(c->histBits.p, 0, cap / 8ull, s), "clearing the per-history table");
    c->histCap = cap;
  }
  // sort the rays as vrc_cast_rays does, the history ids with them
  if (c->opt.sort == 1 || (c->opt.sort == -1 && rp.n >= kAutoSortMin)) {
    VRC_CUDA(c->histSorted.ensure(sizeof(uint32_t) * (size_t)rp.n), "allocating the sorted history ids");
    uint32_t *sorted = static_cast<uint32_t *>(c->histSorted.p);
    int rc = sort_rays(c, rp, s, hist, sorted);
    if (rc) return rc;
    hist = sorted;
  }
  CastArgs a = make_args(c, rp);
  a.hist = hist;
  a.htab.e = static_cast<unsigned long long *>(c->histTab.p);
  a.htab.mask = cap - 1;
  a.htab.bits = static_cast<unsigned int *>(c->histBits.p);
  const int form = c->opt.form;
  const int block = c->opt.block > 0 ? c->opt.block : 256;
  int bps = c->opt.blocks_per_sm;
  if (bps <= 0) {
    VRC_CUDA(cast_hist_occupancy(form, a, block, &bps), "querying occupancy");
    if (bps <= 0) return fail(VRC_ERR_ARG, "cast kernel does not fit on an SM with %d materials", c->n_materials);
  }
  const int grid = (int)std::min<int64_t>((rp.n + block - 1) / block, (int64_t)c->num_sms * bps);
  VRC_CUDA(launch_cast_hist(form, a, grid, block, s), "launching the per-history cast");
  VRC_CUDA(launch_hist_drain(a.htab, static_cast<double *>(c->momS1.p), static_cast<double *>(c->momS2.p),
                             c->num_sms, s),
           "launching the per-history fold");
  c->batches += n_histories;
  return VRC_OK;
}

int vrc_moments_read(vrc_ctx *c, double *total, double *sigma, int64_t n, int64_t *batches,
                     void *cuda_stream) {
  if (!c || !total) return fail(VRC_ERR_ARG, "bad arguments");
  if (!c->moments) return fail(VRC_ERR_STATE, "moments are not enabled");
  const int64_t N = c->ncells * c->n_groups;
  if (n != N) return fail(VRC_ERR_ARG, "moment arrays have %lld entries, caller gave %lld", (long long)N, (long long)n);
  DeviceGuard g(c->device);
  int rc = sync_streams(c, cuda_stream);
  if (rc) return rc;
  VRC_CUDA(cudaMemcpy(total, c->momS1.p, sizeof(double) * N, cudaMemcpyDeviceToHost), "reading S1");
  if (sigma) {
    if (c->batches < 2) {
      std::memset(sigma, 0, sizeof(double) * N);
    } else {
      const int64_t chunk = std::min<int64_t>(N, (int64_t)8 << 20);
      VRC_CUDA(c->scratch.ensure(sizeof(double) * chunk), "allocating moment staging");
      for (int64_t off = 0; off < N; off += chunk) {
        const int64_t m = std::min(chunk, N - off);
        VRC_CUDA(launch_moment_sigma(static_cast<double *>(c->momS1.p) + off,
                                     static_cast<double *>(c->momS2.p) + off,
                                     static_cast<double *>(c->scratch.p), m, (double)c->batches, c->stream),
                 "launching the moment finalize");
        VRC_CUDA(cudaMemcpyAsync(sigma + off, c->scratch.p, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream),
                 "reading sigma");
        VRC_CUDA(cudaStreamSynchronize(c->stream), "reading sigma");
      }
    }
  }
  if (batches) *batches = c->batches;
  unsigned st = 0;
  VRC_CUDA(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost), "reading status");
  return (st & kStatusTableFull) ? status_code(kStatusTableFull) : VRC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Next-event (point-detector) estimator.
// ---------------------------------------------------------------------------
extern "C" {

int vrc_detector_flux(vrc_ctx *c, const vrc_rays *r, const double *det_xyz, int32_t n_det,
                      double *out, void *cuda_stream) {
  if (!c || !r || !det_xyz || !out) return fail(VRC_ERR_ARG, "bad arguments");
  if (n_det < 1 || n_det > 64) return fail(VRC_ERR_ARG, "n_det must be in 1..64");
  if (c->rect) return fail(VRC_ERR_ARG, "the next-event estimator takes a uniform mesh");
  if (r->n < 0) return fail(VRC_ERR_ARG, "ray count is negative");
  const int64_t nout = (int64_t)n_det * c->n_groups;
  if ((int64_t)n_det * c->n_groups * 8 > 64 * 1024) return fail(VRC_ERR_ARG, "n_det * n_groups too large");
  for (int i = 0; i < 3 * n_det; ++i)
    if (!std::isfinite(det_xyz[i])) return fail(VRC_ERR_ARG, "detector position is not finite");
  if (r->n > 0 && (!r->x || !r->y || !r->z || !r->E || !r->wt)) return fail(VRC_ERR_ARG, "a ray array is NULL");
  DeviceGuard g(c->device);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", c->device);
  if (c->xs_dirty) {
    int rc = build_xs(c);
    if (rc) { c->xs_dirty = true; return rc; }
  }
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  std::vector<float> pos(3 * (size_t)n_det);
  for (int i = 0; i < 3 * n_det; ++i) pos[i] = (float)det_xyz[i];
  VRC_CUDA(c->detPos.ensure(sizeof(float) * pos.size()), "allocating detectors");
  VRC_CUDA(c->detOut.ensure(sizeof(double) * nout), "allocating detector flux");
  VRC_CUDA(cudaMemcpyAsync(c->detPos.p, pos.data(), sizeof(float) * pos.size(), cudaMemcpyHostToDevice, s),
           "uploading detectors");
  VRC_CUDA(cudaMemsetAsync(c->detOut.p, 0, sizeof(double) * nout, s), "zeroing detector flux");
  RayPtrs rp;
  std::memset(&rp, 0, sizeof rp);
  rp.n = r->n;
  if (r->n > 0) {
    if (r->on_device) {
      rp.x = r->x; rp.y = r->y; rp.z = r->z; rp.u = r->u; rp.v = r->v; rp.w = r->w; rp.E = r->E; rp.wt = r->wt;
    } else {
      const size_t bytes = sizeof(float) * (size_t)r->n;
      VRC_CUDA(c->stage.ensure(8 * bytes), "allocating ray staging");
      float *base = static_cast<float *>(c->stage.p);
      const float *src[5] = {r->x, r->y, r->z, r->E, r->wt};
      const float **dst[5] = {&rp.x, &rp.y, &rp.z, &rp.E, &rp.wt};
      for (int k = 0; k < 5; ++k) {
        float *dk = base + (size_t)k * r->n;
        VRC_CUDA(cudaMemcpyAsync(dk, src[k], bytes, cudaMemcpyHostToDevice, s), "copying rays");
        *dst[k] = dk;
      }
      rp.u = rp.v = rp.w = rp.x;  // directions are not used
    }
    CastArgs a = make_args(c, rp);
    VRC_CUDA(launch_detectors(c->opt.form, a, static_cast<const float *>(c->detPos.p), n_det,
                              static_cast<double *>(c->detOut.p), c->num_sms, s),
             "launching the detector kernel");
  }
  VRC_CUDA(cudaMemcpyAsync(out, c->detOut.p, sizeof(double) * nout, cudaMemcpyDeviceToHost, s), "reading detector flux");
  VRC_CUDA(cudaStreamSynchronize(s), "waiting for the detector kernel");
  unsigned st = 0;
  VRC_CUDA(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost), "reading status");
  if (st & kStatusTraversal) return status_code(st);
  return VRC_OK;
}

}  // extern "C"
