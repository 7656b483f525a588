/*
 * vrc_micro.h - microbenchmarks that measure the hardware roofs the VRC
 * cast runs against on this GPU: scattered float64 atomic adds (the tally
 * update, one per ray-cell segment of Eq. 4) and the float64 / float32
 * arithmetic rates (the plain form evaluates Eq. 4 in float64, Sec. 3).
 * The paper has no counterpart; these only feed the roofline report.
 *
 * Every call launches asynchronously on `cuda_stream` (NULL = default
 * stream) and returns VRC_OK or VRC_ERR_ARG / VRC_ERR_CUDA; the caller times
 * it with events on the same stream.  All pointers are device pointers.
 */
#ifndef VRC_MICRO_H
#define VRC_MICRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* `updates` float64 atomic adds of 1.0 to pseudo-random indices of
 * buf[0..n) (index = splitmix64(update) mod n).  Each address sees
 * updates/n adds on average; buf must be zeroed by the caller to check the
 * total. */
int vrc_micro_red_f64(double *buf, int64_t n, int64_t updates, void *cuda_stream);

/* Arithmetic rate: `threads` threads each run `iters` rounds of 8
 * independent fused multiply-adds and write one value to out[thread].
 * Work = 2 * 8 * iters * threads floating-point operations. */
int vrc_micro_fma_f64(double *out, int64_t threads, int64_t iters, void *cuda_stream);
int vrc_micro_fma_f32(float *out, int64_t threads, int64_t iters, void *cuda_stream);

/* Transcendental rate: `threads` threads each evaluate expm1 on `iters`
 * dependent arguments (4 independent chains per thread), float64 or
 * float32.  Work = 4 * iters * threads evaluations. */
int vrc_micro_expm1_f64(double *out, int64_t threads, int64_t iters, void *cuda_stream);
int vrc_micro_expm1_f32(float *out, int64_t threads, int64_t iters, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VRC_MICRO_H */
