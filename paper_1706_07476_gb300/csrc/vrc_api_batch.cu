// C ABI of the batched form (Sec. 3 generalised to many problems): a plan
// over many contexts, sorted and cast by one persistent kernel, optionally
// captured in a CUDA graph.
#include "vrc_host.h"

using namespace vrc;
using namespace vrc::host;

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
  if (o->rays_per_warp < 0 || o->rays_per_warp > 8192 || (o->rays_per_warp % 32) != 0)
    return fail(VRC_ERR_ARG, "batch rays_per_warp must be 0 or a multiple of 32 up to 8192");
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
                             b->grid, b->block, b->opt.rays_per_warp, s);
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  cudaError_t e = dev_malloc((void **)dst, sizeof(T) * std::max<size_t>(src.size(), 1));
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
  opt->rays_per_warp = 0;
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
        (e = dev_malloc((void **)&b->d_keys, sizeof(uint32_t) * T)) != cudaSuccess ||
        (e = dev_malloc((void **)&b->d_table, sizeof(uint32_t) * std::max<int64_t>(table, 1))) != cudaSuccess ||
        (e = dev_malloc((void **)&b->d_offsets, sizeof(uint32_t) * std::max<int64_t>(table, 1))) != cudaSuccess ||
        (e = dev_malloc((void **)&b->d_tiles, sizeof(uint32_t) * std::max(b->bplan.n_tiles, 1))) != cudaSuccess ||
        (e = dev_malloc((void **)&b->d_sorted, 8 * sizeof(float) * T)) != cudaSuccess)
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
      (e = dev_malloc((void **)&b->d_queue, sizeof(unsigned int))) != cudaSuccess)
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
