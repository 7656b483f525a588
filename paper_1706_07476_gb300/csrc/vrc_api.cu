// Host implementation of the libvrc C ABI (include/vrc.h): contexts, the
// cast and its shared steps, tally read-back, options and timing.  The
// batched form, the surrogate, streaming, tally moments and the
// next-event estimator live in vrc_api_*.cu.
#include "vrc_host.h"

using namespace vrc;
using namespace vrc::host;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace vrc {
namespace host {

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
  if (e == cudaErrorMemoryAllocation) {
    // a failed allocation also sits in the runtime's last-error slot, where
    // the next launch check (cudaGetLastError) would take it for its own
    (void)cudaGetLastError();
    return fail(VRC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(VRC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Allocations still to succeed before the armed failure (-1: none armed).
std::atomic<long long> g_fail_countdown{-1};

namespace {
bool injected_failure() {
  long long left = g_fail_countdown.load(std::memory_order_relaxed);
  while (left >= 0) {
    if (g_fail_countdown.compare_exchange_weak(left, left - 1, std::memory_order_relaxed))
      return left == 0;  // this allocation is the armed one (the hook disarms itself)
  }
  return false;
}
}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t pinned_alloc(void **p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}

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
  if (o->rays_per_warp < -1 || o->rays_per_warp > 65536 || (o->rays_per_warp > 0 && o->rays_per_warp % 32))
    return fail(VRC_ERR_ARG, "options.rays_per_warp must be -1, 0 or a multiple of 32 up to 65536");
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
  // auto: in the plain form, and in the FP32 form for casts of 2^23 rays or
  // more, warps take 32 sorted rays at a time from the counter.  The warps
  // then work on one contiguous window of the sorted order, whose group's
  // tally slice stays in L2, and warps that finish early take more rays.
  // Smaller FP32 casts use interleaved rounds, whose warps have too few
  // rounds to drift apart.  Measured (FP32 cast, one box): 2^24 slab256
  // rays 15.9 against 17.1 ms interleaved (18.3 ms for chunks of 64),
  // graded 42.3 against 51.1 ms, pin lattice 33.1 against 38.3 ms; 2^22
  // rays 4.50 against 4.36 ms, 2^20 rays 1.29 against 1.21 ms.  Plain form:
  // 2 % faster than interleaved at 2^24 rays.
  a.rays_per_warp = c->opt.rays_per_warp > 0 ? c->opt.rays_per_warp
                    : (c->opt.rays_per_warp == 0 &&
                       (c->opt.form == VRC_FORM_PLAIN || rays.n >= kAutoChunkMinRays) ? 32 : 0);
  a.queue = c->d_queue;
  a.counters = c->d_counters;
  a.status = c->d_status;
  return a;
}

int status_code(unsigned st) {
  if (st & kStatusTimeout)
    return fail(VRC_ERR_CUDA, "a bounded wait on the tensor cores gave up; results are incomplete");
  if (st & kStatusTableFull)
    return fail(VRC_ERR_OOM, "the per-history pairs overflowed their room; their scores are incomplete");
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


// The sort key's layout for this context: (group, crossed-cell bucket),
// accepted-bin rays first when `accepted`, or (group, spatial block).
int sort_key_args(const vrc_ctx *c, bool spatial, bool accepted, SortKeyArgs *out) {
  SortKeyArgs P;
  std::memset(&P, 0, sizeof P);
  for (int k = 0; k < 3; ++k) {
    P.lo[k] = (float)c->org[k];
    P.hi[k] = (float)(c->org[k] + c->n[k] * c->h[k]);
    P.inv_h[k] = (float)(1.0 / c->h[k]);
    P.n[k] = c->n[k];
  }
  P.n_groups = c->n_groups;
  int nl = c->opt.sort_len_buckets > 0 ? c->opt.sort_len_buckets : kAutoLenBuckets;
  while (nl > 1 && (int64_t)c->n_groups * nl + 1 > 16384) nl >>= 1;
  P.n_len = nl;
  const int max_cells = c->n[0] + c->n[1] + c->n[2] + 1;
  P.len_width = std::max(1, (max_cells + nl - 1) / nl);
  P.n_keys = c->n_groups * nl + 1;
  if (accepted) {  // accepted-bin rays first: twice the keys
    while (nl > 1 && 2 * (int64_t)c->n_groups * nl + 1 > 16384) nl >>= 1;
    if (2 * (int64_t)c->n_groups * nl + 1 > 16384)
      return fail(VRC_ERR_ARG, "too many energy groups for the surrogate's sort");
    P.n_len = nl;
    P.len_width = std::max(1, (max_cells + nl - 1) / nl);
    P.n_keys = 2 * c->n_groups * nl + 1;
    P.acc_flags = static_cast<const uint8_t *>(c->mlpFlags.p);
    P.acc_n_hash = c->n_hash;
    P.acc_l2min = c->l2min;
    P.acc_inv_bw = c->inv_bw;
    P.acc_e_lo = c->mlp_lo;
    P.acc_e_hi = c->mlp_hi;
  }
  if (spatial) {  // (group, block) keys on at most 8^3 blocks
    int nb = 8;
    while (nb > 1 && (int64_t)c->n_groups * nb * nb * nb + 1 > 16384) nb >>= 1;
    P.blocks_axis = nb;
    P.n_keys = c->n_groups * nb * nb * nb + 1;
  }
  *out = P;
  return VRC_OK;
}

// Sort scratch for a batch of n rays (grow-only buffers).
int reserve_sort(vrc_ctx *c, const SortPlan &plan) {
  VRC_CUDA(c->sortKeys.ensure(plan.bytes_keys), "allocating sort scratch");
  VRC_CUDA(c->sortTable.ensure(plan.bytes_table), "allocating sort scratch");
  VRC_CUDA(c->sortOffsets.ensure(plan.bytes_table), "allocating sort scratch");
  VRC_CUDA(c->sortTiles.ensure(plan.bytes_tiles), "allocating sort scratch");
  VRC_CUDA(c->sortRays.ensure(plan.bytes_rays), "allocating sort scratch");
  return VRC_OK;
}

int sort_rays(vrc_ctx *c, RayPtrs &rp, cudaStream_t s, const uint32_t *carry_in, uint32_t *carry_out,
              bool spatial, const uint32_t **n_accepted) {
  SortKeyArgs P;
  {
    int rc = sort_key_args(c, spatial, n_accepted != nullptr, &P);
    if (rc) return rc;
  }
  SortPlan plan = make_sort_plan(rp.n, P.n_keys);
  {
    int rc = reserve_sort(c, plan);
    if (rc) return rc;
  }
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
  // the exclusive prefix sum of the (key, chunk) counts at the first key of
  // the not-accepted half is the number of accepted rays
  if (n_accepted)
    *n_accepted = static_cast<const uint32_t *>(c->sortOffsets.p) + (int64_t)c->n_groups * P.n_len * plan.n_chunks;
  return VRC_OK;
}

// With the learned surrogate the rays are always sorted: those in accepted
// energy bins first, so the network runs on exactly that leading range.
bool cast_uses_surrogate(const vrc_ctx *c) { return c->xs_mode == VRC_XS_SURROGATE && c->mlp_ready; }
bool cast_sorts(const vrc_ctx *c, int64_t n) {
  return cast_uses_surrogate(c) || c->opt.sort == 1 || (c->opt.sort == -1 && n >= kAutoSortMin);
}

// Sizes the scratch that cast_device takes for a batch of n rays (sort
// scratch, the surrogate's cross sections), so that casts of up to n rays
// that follow allocate nothing.
int reserve_cast(vrc_ctx *c, int64_t n) {
  const bool surr = cast_uses_surrogate(c);
  if (cast_sorts(c, n)) {
    SortKeyArgs P;
    int rc = sort_key_args(c, false, surr, &P);
    if (rc) return rc;
    rc = reserve_sort(c, make_sort_plan(n, P.n_keys));
    if (rc) return rc;
  }
  if (surr) VRC_CUDA(c->sigBuf.ensure(sizeof(float) * 16 * (size_t)n), "allocating surrogate scratch");
  return VRC_OK;
}

// Sort (optional), surrogate (optional) and cast of a device batch on stream s.
int cast_device(vrc_ctx *c, RayPtrs rp, cudaStream_t s) {
  const bool surr = cast_uses_surrogate(c);
  const bool do_sort = cast_sorts(c, rp.n);
  const uint32_t *n_acc = nullptr;
  if (do_sort) {
    int rc = sort_rays(c, rp, s, nullptr, nullptr, false, surr ? &n_acc : nullptr);
    if (rc) return rc;
  }
  const float *sig_ray = nullptr;
  if (surr) {
    VRC_CUDA(c->sigBuf.ensure(sizeof(float) * 16 * (size_t)rp.n), "allocating surrogate scratch");
    mlp::ApplyArgs aa;
    std::memset(&aa, 0, sizeof aa);
    aa.params = static_cast<const float *>(c->mlpParams.p);
    aa.aos = rp.aos;
    aa.n = rp.n;
    aa.n_limit = n_acc;
    aa.out = static_cast<float *>(c->sigBuf.p);
    aa.mode = 1;
    aa.mat_mask = c->mlp_mask;
    aa.emb = mlp::make_embed(c->mlp_lo, c->mlp_hi);
    aa.status = c->d_status;
    VRC_CUDA(mlp::launch_apply(aa, c->num_sms, s), "launching the surrogate");
    sig_ray = aa.out;
  }
  CastArgs a = make_args(c, rp);
  a.sig_ray = sig_ray;
  a.n_surr = n_acc;
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
  if (a.rays_per_warp > 0)
    VRC_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s), "zeroing the ray counter");
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

}  // namespace host
}  // namespace vrc

void vrc::note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

// Host batches above 2 kFirstChunk rays are uploaded and cast chunk by
// chunk: a small first chunk (only its upload is not overlapped), then
// chunks of up to kUploadChunk.  Few, long casts: each launch ends in a tail
// of long rays, so a 2^24-ray batch in two chunks (2^21, then the rest) ran
// 2 % faster end to end than in three (2^21, 2^23, the rest) on GB300.
constexpr int64_t kUploadChunk = (int64_t)1 << 24;
constexpr int64_t kFirstChunk = (int64_t)1 << 21;

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
  // every buffer the chunks' casts need, before the first of them is
  // launched: an allocation failure then leaves the tally untouched
  {
    const int64_t largest = std::min(kUploadChunk, std::max(kFirstChunk, r->n - kFirstChunk));
    int rc = reserve_cast(c, largest);
    if (rc) return rc;
  }
  const float *src[8] = {r->x, r->y, r->z, r->u, r->v, r->w, r->E, r->wt};
  int last = 0;
  for (int64_t off = 0, i = 0, m = 0; off < r->n; off += m, ++i) {
    const int slot = (int)(i & 1);
    m = std::min(i == 0 ? kFirstChunk : kUploadChunk, r->n - off);
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

}  // namespace

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
  opt->rays_per_warp = 0;
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
  if ((e = dev_malloc((void **)&c->d_mat, (size_t)ncells)) != cudaSuccess ||
      (e = dev_malloc((void **)&c->d_tally, tally_bytes)) != cudaSuccess ||
      (e = dev_malloc((void **)&c->d_counters, sizeof(unsigned long long) * kNumCounters)) != cudaSuccess ||
      (e = dev_malloc((void **)&c->d_status, sizeof(unsigned))) != cudaSuccess ||
      (e = dev_malloc((void **)&c->d_queue, sizeof(unsigned long long))) != cudaSuccess)
    return bail(cuda_fail(e, "allocating the mesh and tally"));
  if (d->group_edges &&
      (e = dev_malloc((void **)&c->d_edges, sizeof(double) * (d->n_groups + 1))) != cudaSuccess)
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
  if (!r->on_device && r->n > 2 * kFirstChunk) return cast_host_pipelined(c, r, s);
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
    stats->live = (int64_t)cnt[kCntLive];
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

int vrc_debug_fail_alloc(int64_t n) {
  g_fail_countdown.store(n < 0 ? -1 : (long long)n, std::memory_order_relaxed);
  return VRC_OK;
}

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
  int nl = c->opt.sort_len_buckets > 0 ? c->opt.sort_len_buckets : kAutoLenBuckets;
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
