// Learned cross-section surrogate: network shape, parameter layout and
// kernel launchers (implementation in vrc_mlp.cu).
//
// The network maps one energy to log Sigma_t of up to 16 materials:
//   x = (log10 E - l0) * inv_range,  features sin(pi f_k x), cos(pi f_k x),
//   f_k = 2^(5k/31), k = 0..31 (64 features, interleaved sin/cos);
//   h1 = silu(W1 x + b1) (64 -> 128), h2 = silu(W2 h1 + b2) (128 -> 128),
//   y = W3 h2 + b3 + log(a + b E^(-1/2)) (128 -> 16).
// The last term is a fixed per-material prior, the 1/v shape of a total
// cross section (a_m > 0, b_m >= 0, fitted to the table before training and
// not trained); the network learns the rest.
// Parameters are float32 masters in one array: W1 [128][64], b1, W2
// [128][128], b2, W3 [16][128], b3, C [16][2] (a_m, b_m).  W1 and W2 are
// rounded to bfloat16 and run on the tensor cores (tcgen05 in the forward
// pass, mma.sync in training) with float32 accumulation; their inputs (the
// features and h1) enter as a pair of bfloat16 values, hi = bf16(v) and
// lo = bf16(v - hi), two products into one accumulator, so the activations
// keep about 16 significant bits (a single bfloat16 rounding, 2^-9, puts
// about 1e-3 of noise on log sigma, the accepted error of the surrogate).
// The 128 -> 16 output layer: in training, float32 on the CUDA cores; in the
// forward pass (vrc_mlp_tc.cu), on the tensor cores with h2 as a bfloat16
// pair and W3 as three bfloat16 parts (hi, mid, lo; about 24 bits), five
// products into one float32 accumulator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vrc {
namespace mlp {

constexpr int kFreq = 32;
constexpr double kFreqMaxLog2 = 5.0;  // highest embedding frequency 2^5
constexpr int kEmb = 64;
constexpr int kHid = 128;
constexpr int kOut = 16;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kEmb;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kOut * kHid;
constexpr int kOffC = kOffB3 + kOut;     // prior coefficients (a_m, b_m)
constexpr int kParams = kOffC + 2 * kOut;  // 26,928
constexpr int kTrained = kOffC;          // Adam updates parameters [0, kTrained)

struct Embed {
  float l0, inv_range;   // x = (log10 E - l0) * inv_range
  float freq[kFreq];     // f_k
};

Embed make_embed(double e_lo, double e_hi);

// Training step on rows of (E, target): forward, loss, backward; adds the
// gradient of the mean squared error (over unmasked (row, material) pairs,
// normalised by inv_count) to grad and the summed squared error times
// inv_count to *loss.  With set_n > 0 the rows are drawn from a training
// set instead: row i uses set entry splitmix64(seed + i) mod set_n.
struct TrainArgs {
  const float *params;
  const float *E;        // [m] (or the training set's energies)
  const float *target;   // [m][16] log sigma (or the training set's)
  const uint8_t *mask;   // [m][16] or nullptr (then mat_mask applies)
  uint32_t mat_mask;     // bit j: output j is trained
  int64_t m;             // rows in this step
  int64_t set_n;         // 0, or the training-set size to sample from
  uint64_t seed;
  float inv_count;
  float *grad;           // [kParams], accumulated
  float *loss;           // scalar, accumulated
  Embed emb;
};

cudaError_t launch_train(const TrainArgs &a, cudaStream_t s);

// Adam (Kingma & Ba) on the float32 masters with bias correction.
cudaError_t launch_adam(float *params, const float *grad, float *m1, float *m2, int n, float lr,
                        float beta1, float beta2, float eps, int step, cudaStream_t s);

// Forward pass for n energies.  mode 0: y = log sigma to out[n][16].
// mode 1: sigma = (a + b E^(-1/2)) exp(W3 h2 + b3) to out[n][16]; outputs
// with bit j clear in mat_mask are written as 0.  With flags set, out[i][0]
// = NaN when the ray's hash bin is flagged (flags[bin] != 0) or its energy
// lies outside [e_first, e_last].  With n_limit set, only rows below
// min(n, *n_limit) are evaluated (a device count, read by the kernel).
struct ApplyArgs {
  const float *params;
  const float *E;          // energies, or nullptr when aos is set
  const float4 *aos;       // 32-byte ray records (E is the third field of the second float4)
  int64_t n;
  float *out;
  int mode;
  uint32_t mat_mask;
  const uint8_t *flags;
  int n_hash;
  float l2min, inv_bw;
  double e_first, e_last;
  Embed emb;
  const uint32_t *n_limit; // device row count to evaluate, or nullptr (all n rows)
  unsigned int *status;    // kStatusTimeout is set here if a tensor-core wait gives up (may be nullptr)
};

// The two 128-wide layers run on tcgen05 (vrc_mlp_tc.cu).  A bounded wait
// on the tensor cores that gives up sets kStatusTimeout in *status and leaves
// the rest of the outputs unwritten.
cudaError_t launch_apply(const ApplyArgs &a, int num_sms, cudaStream_t s);

}  // namespace mlp
}  // namespace vrc
