// C ABI of the streaming ray buffers (Secs. 2-3): pinned buffers filled by
// the caller while earlier ones upload and cast.
#include "vrc_host.h"

using namespace vrc;
using namespace vrc::host;

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
    if ((e = pinned_alloc((void **)&st->host[i], bytes)) != cudaSuccess)
      return bail(e, "allocating a pinned ray buffer");
    if ((e = dev_malloc(&st->dev[i], bytes)) != cudaSuccess) return bail(e, "allocating a device ray buffer");
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
