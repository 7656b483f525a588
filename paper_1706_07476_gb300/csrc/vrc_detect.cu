// Next-event (point-detector) estimator: the flux that every ray event sends
// straight to each detector point, wt exp(-tau)/(4 pi R^2) for isotropic
// emission, tau from the event to the detector through the mesh.  The paper
// names moving this estimator to the GPU as future work (Sec. 6); it reuses
// the cast's cross-section lookup and grid walk.
#include "vrc_device.cuh"

namespace vrc {

namespace {

constexpr float kInv4Pi = 0.0795774715459476678f;  // 1 / (4 pi)
// Optical depths past which exp(-tau) is exactly 0: e^-750 is below half the
// smallest float64 subnormal (e^-744.4) and e^-110 below half the smallest
// float32 subnormal (e^-103.3); the walk to a detector stops there.
constexpr float kTauZeroF64 = 750.f;
constexpr float kTauZeroF32 = 110.f;

template <int FORM>
__global__ void __launch_bounds__(256) k_detectors(CastArgs a, const float *__restrict__ det, int n_det,
                                                   double *__restrict__ out, size_t hash_off, size_t acc_off,
                                                   size_t sig_off) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *hash_s = reinterpret_cast<int32_t *>(smem + hash_off);
  double *acc = reinterpret_cast<double *>(smem + acc_off);  // [n_det][n_groups]
  float *sig_s = reinterpret_cast<float *>(smem + sig_off) + threadIdx.x;
  float *inv_s = sig_s + (size_t)a.xs.n_mat * blockDim.x;  // 1/sigma (unused here)
  const int G = a.n_groups;
  if (a.xs.n_union > 0)
    for (int t = threadIdx.x; t <= a.xs.n_hash; t += blockDim.x) hash_s[t] = a.xs.hash[t];
  for (int t = threadIdx.x; t < n_det * G; t += blockDim.x) acc[t] = 0.0;
  __syncthreads();
  const int stride = blockDim.x;
  bool ovf = false;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.rays.n;
       r += (int64_t)gridDim.x * blockDim.x) {
    float f[8];
    load_ray(a.rays, r, f);
    if (!(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]) && isfinite(f[6]) && isfinite(f[7]) &&
          f[6] > 0.f))
      continue;
    const int g = group_of(a.edges, G, (double)f[6]);
    if (g < 0) continue;
    xs_lookup(a.xs, hash_s, f[6], sig_s, inv_s, stride);
    const float p[3] = {f[0], f[1], f[2]};
    for (int k = 0; k < n_det; ++k) {
      const float q[3] = {det[3 * k], det[3 * k + 1], det[3 * k + 2]};
      const float R2 = (q[0] - p[0]) * (q[0] - p[0]) + (q[1] - p[1]) * (q[1] - p[1]) + (q[2] - p[2]) * (q[2] - p[2]);
      if (!(R2 > 0.f)) continue;
      const df tau = optical_depth(a.mesh, p, q, sig_s, stride,
                                   FORM == kFormPlain ? kTauZeroF64 : kTauZeroF32, &ovf);
      double v;
      if (FORM == kFormPlain)
        v = (double)f[7] * exp(-((double)tau.hi + (double)tau.lo)) * (double)kInv4Pi / (double)R2;
      else
        v = (double)(f[7] * expf(-tau.hi) * (1.f - tau.lo) * kInv4Pi / R2);
      if (v != 0.0) atomicAdd(acc + k * G + g, v);
    }
  }
  if (ovf) atomicOr(a.status, kStatusTraversal);
  __syncthreads();
  for (int t = threadIdx.x; t < n_det * G; t += blockDim.x)
    if (acc[t] != 0.0) atomicAdd(out + t, acc[t]);
}

}  // namespace

cudaError_t launch_detectors(int form, const CastArgs &a, const float *det, int n_det, double *out,
                             int num_sms, cudaStream_t s) {
  if (a.rays.n <= 0 || n_det <= 0) return cudaSuccess;
  const int block = 256;
  size_t off = 0;
  const size_t hash_off = off;
  off += sizeof(int32_t) * ((size_t)(a.xs.n_union > 0 ? a.xs.n_hash : 0) + 1);
  off = (off + 15) / 16 * 16;
  const size_t acc_off = off;
  off += sizeof(double) * (size_t)n_det * a.n_groups;
  off = (off + 15) / 16 * 16;
  const size_t sig_off = off;
  off += 2 * sizeof(float) * (size_t)a.xs.n_mat * block;
  const size_t smem = (off + 15) / 16 * 16;
  cudaError_t e;
  if (form == kFormPlain) {
    if ((e = cudaFuncSetAttribute(k_detectors<kFormPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  } else {
    if ((e = cudaFuncSetAttribute(k_detectors<kFormFp32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  }
  const int64_t need = (a.rays.n + block - 1) / block;
  const int grid = (int)(need < (int64_t)num_sms * 4 ? need : (int64_t)num_sms * 4);
  if (form == kFormPlain)
    k_detectors<kFormPlain><<<grid, block, smem, s>>>(a, det, n_det, out, hash_off, acc_off, sig_off);
  else
    k_detectors<kFormFp32><<<grid, block, smem, s>>>(a, det, n_det, out, hash_off, acc_off, sig_off);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace vrc
