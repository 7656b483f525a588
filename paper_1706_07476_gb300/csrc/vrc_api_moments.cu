// C ABI of the tally moments (the sigma of Eqs. 5 and 8): batch folds,
// per-history casts and the read-back of total and sigma.
#include "vrc_host.h"

using namespace vrc;
using namespace vrc::host;

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
    c->mom.release();
    c->pairBuf.release();
    c->pairSorted.release();
    c->moments = false;
    return VRC_OK;
  }
  const size_t bytes = sizeof(double2) * (size_t)(c->ncells * c->n_groups);
  VRC_CUDA(c->mom.ensure(bytes), "allocating tally moments");
  VRC_CUDA(cudaMemsetAsync(c->mom.p, 0, bytes, c->stream), "zeroing tally moments");
  c->moments = true;
  return VRC_OK;
}

int vrc_moments_fold(vrc_ctx *c, void *cuda_stream) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  if (!c->moments) return fail(VRC_ERR_STATE, "moments are not enabled");
  if (c->moment_mode != VRC_MOMENTS_BATCH) return fail(VRC_ERR_STATE, "moments are per history, not per batch");
  DeviceGuard g(c->device);
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  VRC_CUDA(launch_fold_moments(c->d_tally, static_cast<double2 *>(c->mom.p), c->ncells * c->n_groups, s),
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
  // sort the rays as vrc_cast_rays does, the history ids with them
  if (c->opt.sort == 1 || (c->opt.sort == -1 && rp.n >= kAutoSortMin)) {
    VRC_CUDA(c->histSorted.ensure(sizeof(uint32_t) * (size_t)rp.n), "allocating the sorted history ids");
    uint32_t *sorted = static_cast<uint32_t *>(c->histSorted.p);
    int rc = sort_rays(c, rp, s, hist, sorted);
    if (rc) return rc;
    hist = sorted;
  }
  const size_t nr = (size_t)rp.n;
  VRC_CUDA(c->rayCnt.ensure(sizeof(uint32_t) * nr), "allocating per-ray pair counts");
  const int tile = scan_tile_elems();
  // buckets of 2^shift consecutive bins, at most kPairMaxBuckets of them
  const int64_t n_bins = c->ncells * c->n_groups;
  int shift = 0;
  while (((n_bins - 1) >> shift) + 1 > kPairMaxBuckets) ++shift;
  const int n_buckets = (int)(((n_bins - 1) >> shift) + 1);
  const int64_t tiles = std::max<int64_t>(((int64_t)n_buckets + tile) / tile, ((int64_t)nr + tile - 1) / tile);
  VRC_CUDA(c->pairBoff.ensure(sizeof(uint32_t) * 2 * (size_t)(n_buckets + 1)), "allocating the pair sort table");
  VRC_CUDA(c->pairTiles.ensure(sizeof(uint32_t) * (size_t)tiles), "allocating the pair sort table");

  // Each ray's stretch of the pair buffer.  With device inputs, a fixed
  // stretch of nx + ny + nz + 10 pairs per ray (more than any walk's
  // segments) when two such buffers fit in a quarter of the free device
  // memory: no per-ray bound is needed and the call never waits on the
  // device (it synchronises the stream only when it grows the buffers).
  // Otherwise (or with host inputs, which must be free on return) each
  // ray's room is an upper bound of its segments, the stretches follow by a
  // scan, and the call reads the total back to size the buffers.
  const uint32_t stride = (uint32_t)(c->n[0] + c->n[1] + c->n[2] + 10);
  const unsigned long long worst = (unsigned long long)nr * stride;
  bool fixed = false;
  if (r->on_device && worst < 0xffffffffull) {
    const size_t wbytes = 16ull * worst;
    if (wbytes <= c->pairBuf.bytes && wbytes <= c->pairSorted.bytes) {
      fixed = true;
    } else {
      size_t free_b = 0, total_b = 0;
      VRC_CUDA(cudaStreamSynchronize(s), "waiting for earlier work on the pair buffers");
      VRC_CUDA(cudaMemGetInfo(&free_b, &total_b), "querying device memory");
      if (2 * wbytes <= (free_b + c->pairBuf.bytes + c->pairSorted.bytes) / 4) {
        c->pairBuf.release();
        c->pairSorted.release();
        VRC_CUDA(c->pairBuf.ensure(wbytes), "allocating the pair buffer");
        VRC_CUDA(c->pairSorted.ensure(wbytes), "allocating the pair buffer");
        fixed = true;
      }
    }
  }
  uint32_t *cap = nullptr, *off = nullptr;
  if (!fixed) {
    BoundGeom G;
    for (int k = 0; k < 3; ++k) {
      G.lo[k] = c->org[k];
      G.h[k] = c->h[k];
      G.n[k] = c->n[k];
      G.e[k] = c->rect ? static_cast<const double *>(c->rectD.p) + c->rect_off[k] : nullptr;
    }
    VRC_CUDA(c->rayCap.ensure(sizeof(uint32_t) * nr), "allocating per-ray pair room");
    VRC_CUDA(c->rayOff.ensure(sizeof(uint32_t) * nr), "allocating per-ray pair room");
    cap = static_cast<uint32_t *>(c->rayCap.p);
    off = static_cast<uint32_t *>(c->rayOff.p);
    VRC_CUDA(launch_ray_caps(G, rp, cap, c->num_sms, s), "launching the pair room");
    VRC_CUDA(launch_exclusive_scan(cap, rp.n, off, static_cast<uint32_t *>(c->pairTiles.p), s),
             "launching the pair room scan");
    VRC_CUDA(c->histBound.ensure(2 * sizeof(uint32_t)), "allocating the pair count");
    uint32_t *d_last = static_cast<uint32_t *>(c->histBound.p);
    VRC_CUDA(cudaMemcpyAsync(d_last, cap + nr - 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s), "reading the pair room");
    VRC_CUDA(cudaMemcpyAsync(d_last + 1, off + nr - 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s), "reading the pair room");
    uint32_t last[2] = {0, 0};
    VRC_CUDA(cudaMemcpyAsync(last, d_last, sizeof last, cudaMemcpyDeviceToHost, s), "reading the pair room");
    VRC_CUDA(cudaStreamSynchronize(s), "waiting for the pair room");  // host arrays are free from here
    const unsigned long long total = (unsigned long long)last[0] + last[1];
    if (total >= 0xffffffffull)
      return fail(VRC_ERR_OOM, "this call's rays may cross up to %llu cells, more than 2^32 - 1; split the call",
                  total);
    const size_t pair_bytes = 16ull * std::max<unsigned long long>(total, 1);
    if (pair_bytes > c->pairBuf.bytes || pair_bytes > c->pairSorted.bytes) {
      c->pairBuf.release();
      c->pairSorted.release();
      size_t free_b = 0, total_b = 0;
      VRC_CUDA(cudaMemGetInfo(&free_b, &total_b), "querying device memory");
      if (2 * pair_bytes > free_b / 10 * 9)
        return fail(VRC_ERR_OOM, "this call's histories need %.1f GB of pair buffers (%.1f GB free); split the call",
                    2 * pair_bytes / 1e9, free_b / 1e9);
      VRC_CUDA(c->pairBuf.ensure(pair_bytes), "allocating the pair buffer");
      VRC_CUDA(c->pairSorted.ensure(pair_bytes), "allocating the pair buffer");
    }
  }
  CastArgs a = make_args(c, rp);
  a.hist = hist;
  a.pout.pairs = static_cast<ulonglong2 *>(c->pairBuf.p);
  a.pout.off = off;
  a.pout.cap = cap;
  a.pout.stride = fixed ? stride : 0u;
  a.pout.cnt = static_cast<uint32_t *>(c->rayCnt.p);
  uint32_t *bcount = static_cast<uint32_t *>(c->pairBoff.p), *bbase = bcount + (n_buckets + 1);
  a.pout.bcount = bcount;
  a.pout.bshift = shift;
  VRC_CUDA(cudaMemsetAsync(bcount, 0, sizeof(uint32_t) * (size_t)(n_buckets + 1), s), "zeroing the bucket counts");
  // rays the cast rejects write no count
  VRC_CUDA(cudaMemsetAsync(a.pout.cnt, 0, sizeof(uint32_t) * nr, s), "zeroing the pair counts");
  const int form = c->opt.form;
  const int block = c->opt.block > 0 ? c->opt.block : 256;
  int bps = c->opt.blocks_per_sm;
  if (bps <= 0) {
    VRC_CUDA(cast_hist_occupancy(form, a, block, &bps), "querying occupancy");
    if (bps <= 0) return fail(VRC_ERR_ARG, "cast kernel does not fit on an SM with %d materials", c->n_materials);
  }
  const int grid = (int)std::min<int64_t>((rp.n + block - 1) / block, (int64_t)c->num_sms * bps);
  if (a.rays_per_warp > 0)
    VRC_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s), "zeroing the ray counter");
  VRC_CUDA(launch_cast_hist(form, a, grid, block, s), "launching the per-history cast");
  VRC_CUDA(launch_pair_fold(a.pout, rp.n, n_buckets, bbase, static_cast<uint32_t *>(c->pairTiles.p),
                            static_cast<ulonglong2 *>(c->pairSorted.p), static_cast<double2 *>(c->mom.p),
                            c->d_status, c->num_sms, s),
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
  // S1 (and sigma) by chunks of 8 Mi bins through device staging
  const bool want_sigma = sigma && c->batches >= 2;
  if (sigma && !want_sigma) std::memset(sigma, 0, sizeof(double) * N);
  const int64_t chunk = std::min<int64_t>(N, (int64_t)8 << 20);
  VRC_CUDA(c->scratch.ensure(2 * sizeof(double) * chunk), "allocating moment staging");
  double *st_total = static_cast<double *>(c->scratch.p), *st_sigma = st_total + chunk;
  for (int64_t off = 0; off < N; off += chunk) {
    const int64_t m = std::min(chunk, N - off);
    VRC_CUDA(launch_moment_read(static_cast<const double2 *>(c->mom.p) + off, st_total,
                                want_sigma ? st_sigma : nullptr, m, (double)c->batches, c->stream),
             "launching the moment read");
    VRC_CUDA(cudaMemcpyAsync(total + off, st_total, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream),
             "reading S1");
    if (want_sigma)
      VRC_CUDA(cudaMemcpyAsync(sigma + off, st_sigma, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream),
               "reading sigma");
    VRC_CUDA(cudaStreamSynchronize(c->stream), "reading moments");
  }
  if (batches) *batches = c->batches;
  unsigned st = 0;
  VRC_CUDA(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost), "reading status");
  return (st & kStatusTableFull) ? status_code(kStatusTableFull) : VRC_OK;
}

}  // extern "C"
