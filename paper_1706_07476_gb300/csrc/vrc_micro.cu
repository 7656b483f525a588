// Microbenchmarks for the roofline report (include/vrc_micro.h).
#include <stdint.h>

#include "vrc.h"
#include "vrc_internal.h"
#include "vrc_micro.h"

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_red_f64(double *buf, int64_t n, int64_t updates) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < updates;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(buf + (int64_t)(splitmix64((uint64_t)i) % (uint64_t)n), 1.0);
}

template <typename T>
__global__ void k_fma(T *out, int64_t threads, int64_t iters) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= threads) return;
  T a[8];
  const T m = (T)0.999999, c = (T)1e-7;
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (T)(t + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[t] = s;
}

template <typename T>
__device__ __forceinline__ T expm1_t(T x);
template <>
__device__ __forceinline__ double expm1_t<double>(double x) { return expm1(x); }
template <>
__device__ __forceinline__ float expm1_t<float>(float x) { return expm1f(x); }

template <typename T>
__global__ void k_expm1(T *out, int64_t threads, int64_t iters) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= threads) return;
  T a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = (T)(-1e-3 * (double)((t + k) & 1023));
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = (T)(-0.5) * expm1_t<T>(a[k]) - (T)0.25;
  }
  out[t] = a[0] + a[1] + a[2] + a[3];
}

int launch_status(const char *) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

int grid_for(int64_t threads, int block) { return (int)((threads + block - 1) / block); }

}  // namespace

extern "C" {

int vrc_micro_red_f64(double *buf, int64_t n, int64_t updates, void *stream) {
  if (!buf || n <= 0 || updates < 0) return VRC_ERR_ARG;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_red_f64<<<sms * 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(buf, n, updates);
  vrc::note_launches(1);
  return launch_status("red");
}

int vrc_micro_fma_f64(double *out, int64_t threads, int64_t iters, void *stream) {
  if (!out || threads <= 0 || threads > ((int64_t)1 << 31) || iters < 0) return VRC_ERR_ARG;
  k_fma<double><<<grid_for(threads, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(out, threads, iters);
  vrc::note_launches(1);
  return launch_status("fma64");
}

int vrc_micro_fma_f32(float *out, int64_t threads, int64_t iters, void *stream) {
  if (!out || threads <= 0 || threads > ((int64_t)1 << 31) || iters < 0) return VRC_ERR_ARG;
  k_fma<float><<<grid_for(threads, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(out, threads, iters);
  vrc::note_launches(1);
  return launch_status("fma32");
}

int vrc_micro_expm1_f64(double *out, int64_t threads, int64_t iters, void *stream) {
  if (!out || threads <= 0 || threads > ((int64_t)1 << 31) || iters < 0) return VRC_ERR_ARG;
  k_expm1<double><<<grid_for(threads, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(out, threads, iters);
  vrc::note_launches(1);
  return launch_status("expm1_64");
}

int vrc_micro_expm1_f32(float *out, int64_t threads, int64_t iters, void *stream) {
  if (!out || threads <= 0 || threads > ((int64_t)1 << 31) || iters < 0) return VRC_ERR_ARG;
  k_expm1<float><<<grid_for(threads, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(out, threads, iters);
  vrc::note_launches(1);
  return launch_status("expm1_32");
}

}  // extern "C"
