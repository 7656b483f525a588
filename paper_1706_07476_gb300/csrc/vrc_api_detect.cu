// C ABI of the next-event (point-detector) estimator (Sec. 6.3).
#include "vrc_host.h"

using namespace vrc;
using namespace vrc::host;

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
    // events sorted by (group, spatial block): the 32 lanes of a warp then
    // walk from nearby points at similar cross sections
    if (c->opt.sort == 1 || (c->opt.sort == -1 && rp.n >= kAutoSortMin)) {
      int rc = sort_rays(c, rp, s, nullptr, nullptr, true);
      if (rc) return rc;
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
