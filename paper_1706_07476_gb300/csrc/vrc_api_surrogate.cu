// C ABI of the learned cross-section surrogate: forward pass and gradient
// entry points, training on the context's own tables, validation and mode.
#include "vrc_host.h"

using namespace vrc;
using namespace vrc::host;

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
    cudaError_t e = dev_malloc(p, std::max<size_t>(bytes, 16));
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
  opt->steps = 12000;
  opt->batch = 4096;
  opt->lr = 5e-3f;
  opt->tol = 1e-3f;
  opt->seed = 4;
  opt->smooth = 5e-6f;
}

int vrc_train_surrogate(vrc_ctx *c, const vrc_surrogate_options *opt, vrc_surrogate_report *report) {
  if (!c) return fail(VRC_ERR_ARG, "context is NULL");
  vrc_surrogate_options o;
  vrc_default_surrogate_options(&o);
  if (opt) o = *opt;
  if (o.steps < 0 || o.batch < 64 || o.batch > (1 << 22) || !(o.lr > 0.f) || !(o.tol > 0.f) ||
      !(o.smooth > 0.f))
    return fail(VRC_ERR_ARG, "bad surrogate options");
  if (c->n_materials > mlp::kOut)
    return fail(VRC_ERR_ARG, "the surrogate models at most %d materials", mlp::kOut);
  DeviceGuard g(c->device);
  if (!g.ok) return fail(VRC_ERR_CUDA, "cannot select CUDA device %d", c->device);
  if (c->xs_dirty) {
    int rc = build_xs(c);
    if (rc) { c->xs_dirty = true; return rc; }
  }
  const bool revalidate = o.steps == 0;
  if (revalidate && !c->mlp_ready) return fail(VRC_ERR_STATE, "no trained surrogate to re-validate");
  uint32_t mask = 0;
  for (int m = 0; m < c->n_materials; ++m)
    if (c->loaded[m] && !c->tabE[m].empty()) mask |= 1u << m;
  if (mask == 0 || c->n_union < 2) return fail(VRC_ERR_STATE, "no cross-section tables to learn");
  // a table with a zero sigma cannot be modelled in log sigma; rays would
  // then need the table for that material, so no bin is accepted at all
  bool unmodelled = false;
  for (int m = 0; m < c->n_materials; ++m)
    if ((mask >> m) & 1u)
      for (double v : c->tabS[m])
        if (!(v > 0.0)) { mask &= ~(1u << m); unmodelled = true; break; }

  std::vector<double> U((size_t)c->n_union);
  VRC_CUDA(cudaMemcpy(U.data(), c->xsE.p, sizeof(double) * U.size(), cudaMemcpyDeviceToHost), "reading the grid");
  const int nm = c->n_materials;
  const size_t nu = U.size();

  // Smooth union-grid points: log sigma of every modelled material deviates
  // from the straight line (in log E) through its two neighbours by less
  // than o.smooth, at the point and at the 3 points on either side.  Only
  // intervals between two smooth points are trained on: a resonance's sharp
  // structure stays with the table, and the network's capacity goes to the
  // parts of the tables it can fit to the bound.
  std::vector<std::vector<double>> LS(nm);  // log sigma at the union points
  for (int m = 0; m < nm; ++m)
    if ((mask >> m) & 1u) {
      LS[m].resize(nu);
      for (size_t i = 0; i < nu; ++i) LS[m][i] = std::log(table_sigma(c->tabE[m], c->tabS[m], U[i]));
    }
  std::vector<double> dev(nu, 0.0);
  for (size_t i = 1; i + 1 < nu; ++i) {
    const double x0 = std::log(U[i - 1]), x1 = std::log(U[i]), x2 = std::log(U[i + 1]);
    for (int m = 0; m < nm; ++m)
      if ((mask >> m) & 1u) {
        const double lin = (LS[m][i - 1] * (x2 - x1) + LS[m][i + 1] * (x1 - x0)) / (x2 - x0);
        dev[i] = std::max(dev[i], std::fabs(LS[m][i] - lin));
      }
  }
  std::vector<uint8_t> smooth(nu, 0);
  for (size_t i = 0; i < nu; ++i) {
    double w = 0.0;
    for (size_t j = (i >= 3 ? i - 3 : 0); j <= std::min(nu - 1, i + 3); ++j) w = std::max(w, dev[j]);
    smooth[i] = w < (double)o.smooth;
  }

  // training energies: fractions 0, 1/4, 1/2, 3/4 of every smooth interval;
  // validation at (k + 1/2)/8 of every interval
  std::vector<float> trE, trT, vaE;
  std::vector<double> vaE64;
  int64_t smooth_intervals = 0;
  for (size_t i = 0; i + 1 < nu; ++i) {
    if (smooth[i] && smooth[i + 1]) {
      ++smooth_intervals;
      for (int q = 0; q < 4; ++q) trE.push_back((float)(U[i] + (U[i + 1] - U[i]) * q / 4.0));
    }
    for (int q = 0; q < 8; ++q) {
      const double e = U[i] + (U[i + 1] - U[i]) * (q + 0.5) / 8.0;
      vaE.push_back((float)e);
      vaE64.push_back((double)(float)e);
    }
  }
  const int64_t n_tr = (int64_t)trE.size(), n_va = (int64_t)vaE.size();

  // the 1/v prior per material: sigma ~ a + b E^(-1/2), least squares in
  // relative error over the smooth points (all points if none), a > 0, b >= 0
  double Cab[mlp::kOut][2];
  for (int m = 0; m < mlp::kOut; ++m) { Cab[m][0] = 1.0; Cab[m][1] = 0.0; }
  for (int m = 0; m < nm; ++m) {
    if (!((mask >> m) & 1u)) continue;
    double s00 = 0, s01 = 0, s11 = 0, r0 = 0, r1 = 0, smin = INFINITY;
    for (int pass = 0; pass < 2 && s00 == 0.0; ++pass)
      for (size_t i = 0; i < nu; ++i) {
        if (pass == 0 && !smooth[i]) continue;
        const double S = std::exp(LS[m][i]), r = 1.0 / std::sqrt(U[i]), w2 = 1.0 / (S * S);
        s00 += w2; s01 += w2 * r; s11 += w2 * r * r; r0 += w2 * S; r1 += w2 * S * r;
        smin = std::min(smin, S);
      }
    const double det = s00 * s11 - s01 * s01;
    double a = r0 / s00, b = 0.0;
    if (det > 0.0) {
      a = (r0 * s11 - r1 * s01) / det;
      b = (s00 * r1 - s01 * r0) / det;
    }
    if (b < 0.0) { b = 0.0; a = r0 / s00; }
    Cab[m][0] = std::max(a, 1e-3 * smin);
    Cab[m][1] = b;
  }
  auto prior = [&](int m, double e) { return Cab[m][0] + Cab[m][1] / std::sqrt(e); };

  // targets: log sigma minus the prior, normalised per material (mean 0,
  // spread 1 over the training set); the normalisation is folded into W3
  // and b3 after training
  double mu[mlp::kOut] = {}, sd[mlp::kOut];
  for (int m = 0; m < mlp::kOut; ++m) sd[m] = 1.0;
  trT.assign((size_t)n_tr * mlp::kOut, 0.f);
  if (n_tr > 0) {
    std::vector<double> t((size_t)n_tr);
    for (int m = 0; m < nm; ++m) {
      if (!((mask >> m) & 1u)) continue;
      double s1 = 0, s2 = 0;
      for (int64_t i = 0; i < n_tr; ++i) {
        t[i] = std::log(table_sigma(c->tabE[m], c->tabS[m], (double)trE[i]) / prior(m, (double)trE[i]));
        s1 += t[i];
        s2 += t[i] * t[i];
      }
      mu[m] = s1 / n_tr;
      sd[m] = std::max(std::sqrt(std::max(s2 / n_tr - mu[m] * mu[m], 0.0)), 1e-3);
      for (int64_t i = 0; i < n_tr; ++i) trT[(size_t)i * mlp::kOut + m] = (float)((t[i] - mu[m]) / sd[m]);
    }
  }

  // initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases;
  // the prior is held at a = 1, b = 0 (log 1 = 0) while training
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
  for (int m = 0; m < mlp::kOut; ++m) P[mlp::kOffC + 2 * m] = 1.f;

  TmpDev tmp;
  float *d_trE = nullptr, *d_trT = nullptr, *d_grad, *d_m1, *d_m2, *d_loss, *d_vaE, *d_vaY;
  VRC_CUDA(tmp.alloc((void **)&d_trE, sizeof(float) * std::max<int64_t>(n_tr, 1)), "allocating training data");
  VRC_CUDA(tmp.alloc((void **)&d_trT, sizeof(float) * std::max<size_t>(trT.size(), 1)), "allocating training data");
  VRC_CUDA(tmp.alloc((void **)&d_grad, sizeof(float) * mlp::kParams), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_m1, sizeof(float) * mlp::kParams), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_m2, sizeof(float) * mlp::kParams), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_loss, sizeof(float) * (o.steps + 1)), "allocating training state");
  VRC_CUDA(tmp.alloc((void **)&d_vaE, sizeof(float) * n_va), "allocating validation data");
  VRC_CUDA(tmp.alloc((void **)&d_vaY, sizeof(float) * n_va * mlp::kOut), "allocating validation data");
  VRC_CUDA(c->mlpParams.ensure(sizeof(float) * mlp::kParams), "allocating the surrogate");
  VRC_CUDA(c->mlpFlags.ensure((size_t)c->n_hash), "allocating the surrogate flags");
  float *d_P = static_cast<float *>(c->mlpParams.p);
  cudaStream_t s = c->stream;
  if (n_tr > 0) {
    VRC_CUDA(cudaMemcpy(d_trE, trE.data(), sizeof(float) * n_tr, cudaMemcpyHostToDevice), "uploading training data");
    VRC_CUDA(cudaMemcpy(d_trT, trT.data(), sizeof(float) * trT.size(), cudaMemcpyHostToDevice), "uploading training data");
  }
  VRC_CUDA(cudaMemcpy(d_vaE, vaE.data(), sizeof(float) * n_va, cudaMemcpyHostToDevice), "uploading validation data");
  VRC_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float) * (o.steps + 1), s), "zeroing losses");
  const int n_out = __builtin_popcount(mask);
  if (!revalidate) {
    VRC_CUDA(cudaMemcpy(d_P, P.data(), sizeof(float) * mlp::kParams, cudaMemcpyHostToDevice), "uploading weights");
    VRC_CUDA(cudaMemsetAsync(d_m1, 0, sizeof(float) * mlp::kParams, s), "zeroing Adam state");
    VRC_CUDA(cudaMemsetAsync(d_m2, 0, sizeof(float) * mlp::kParams, s), "zeroing Adam state");
    mlp::TrainArgs ta;
    std::memset(&ta, 0, sizeof ta);
    ta.params = d_P;
    ta.E = d_trE;
    ta.target = d_trT;
    ta.mat_mask = mask;
    ta.m = o.batch;
    ta.set_n = n_tr;
    ta.inv_count = 1.f / (float)((int64_t)o.batch * std::max(n_out, 1));
    ta.grad = d_grad;
    ta.emb = mlp::make_embed(U.front(), U.back());
    const int warm = std::min(200, std::max(1, o.steps / 20));
    for (int step = 1; step <= o.steps && n_tr > 0 && n_out > 0; ++step) {
      VRC_CUDA(cudaMemsetAsync(d_grad, 0, sizeof(float) * mlp::kParams, s), "zeroing the gradient");
      ta.seed = host_mix64(o.seed ^ ((uint64_t)step << 32));
      ta.loss = d_loss + step;
      VRC_CUDA(mlp::launch_train(ta, s), "launching a training step");
      const double prog = (double)(step - 1) / std::max(1, o.steps - 1);
      double lr = o.lr * (0.02 + 0.98 * 0.5 * (1.0 + std::cos(M_PI * prog)));
      if (step <= warm) lr *= (double)step / warm;
      VRC_CUDA(mlp::launch_adam(d_P, d_grad, d_m1, d_m2, mlp::kTrained, (float)lr, 0.9f, 0.999f, 1e-8f, step, s),
               "launching Adam");
    }
    // fold the target normalisation into W3 and b3, and set the prior
    VRC_CUDA(cudaMemcpyAsync(P.data(), d_P, sizeof(float) * mlp::kParams, cudaMemcpyDeviceToHost, s),
             "reading the trained weights");
    VRC_CUDA(cudaStreamSynchronize(s), "training the surrogate");
    for (int m = 0; m < mlp::kOut; ++m) {
      for (int k = 0; k < mlp::kHid; ++k) P[mlp::kOffW3 + m * mlp::kHid + k] *= (float)sd[m];
      P[mlp::kOffB3 + m] = (float)(sd[m] * P[mlp::kOffB3 + m] + mu[m]);
      P[mlp::kOffC + 2 * m] = (float)Cab[m][0];
      P[mlp::kOffC + 2 * m + 1] = (float)Cab[m][1];
    }
    VRC_CUDA(cudaMemcpy(d_P, P.data(), sizeof(float) * mlp::kParams, cudaMemcpyHostToDevice), "uploading weights");
  }
  // validation: log sigma of the network (prior included) against the tables
  mlp::ApplyArgs aa;
  std::memset(&aa, 0, sizeof aa);
  aa.params = d_P;
  aa.E = d_vaE;
  aa.n = n_va;
  aa.out = d_vaY;
  aa.mode = 0;
  aa.mat_mask = mask;
  aa.emb = mlp::make_embed(U.front(), U.back());
  aa.status = c->d_status;
  VRC_CUDA(mlp::launch_apply(aa, c->num_sms, s), "launching the validation pass");
  std::vector<float> Y((size_t)n_va * mlp::kOut), L((size_t)o.steps + 1, 0.f);
  VRC_CUDA(cudaStreamSynchronize(s), "validating the surrogate");
  VRC_CUDA(cudaMemcpy(Y.data(), d_vaY, sizeof(float) * Y.size(), cudaMemcpyDeviceToHost), "reading validation");
  VRC_CUDA(cudaMemcpy(L.data(), d_loss, sizeof(float) * L.size(), cudaMemcpyDeviceToHost), "reading losses");

  std::vector<float> bin_err((size_t)c->n_hash, 0.f), all_err;
  std::vector<int32_t> bin_pts((size_t)c->n_hash, 0);
  all_err.reserve((size_t)n_va);
  const double l2a = std::log2(U.front());
  for (int64_t i = 0; i < n_va; ++i) {
    float worst = 0.f;
    for (int m = 0; m < nm; ++m) {
      if (!((mask >> m) & 1u)) continue;
      const double sg = table_sigma(c->tabE[m], c->tabS[m], vaE64[i]);
      const double got = std::exp((double)Y[(size_t)i * mlp::kOut + m]);
      const float err = (float)(std::fabs(got - sg) / sg);
      worst = std::isnan(err) ? INFINITY : std::max(worst, err);
    }
    int b = (int)std::floor((std::log2(vaE64[i]) - l2a) * c->inv_bw);
    b = std::min(std::max(b, 0), c->n_hash - 1);
    bin_err[b] = std::max(bin_err[b], worst);
    bin_pts[b] += 1;
    all_err.push_back(worst);
  }
  // a bin is accepted when it and both neighbours were validated within tol
  std::vector<uint8_t> flags((size_t)c->n_hash, 0);
  int accepted = 0;
  float max_acc = 0.f;
  auto bad_bin = [&](int b) { return bin_pts[b] == 0 || !(bin_err[b] <= o.tol); };
  for (int b = 0; b < c->n_hash; ++b) {
    bool bad = unmodelled || bad_bin(b);
    if (b > 0) bad = bad || bad_bin(b - 1);
    if (b + 1 < c->n_hash) bad = bad || bad_bin(b + 1);
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
    report->smooth_fraction = nu > 1 ? (float)smooth_intervals / (float)(nu - 1) : 0.f;
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
