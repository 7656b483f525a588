// Device building blocks of the VRC cast: double-float arithmetic, the
// hashed union-grid cross-section lookup, and the per-ray grid walk with the
// Eq. 4 score.  Included by the cast and batched kernels.
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "vrc_math64.h"
#include "vrc_internal.h"

namespace vrc {

constexpr int kFormPlain = 0;
constexpr int kFormFp32 = 1;

// ---------------------------------------------------------------------------
// Double-float arithmetic: error-free transformations of Knuth (TwoSum) and
// Dekker (Fast2Sum), with the product error taken exactly by one fused
// multiply-add.  The _rn intrinsics keep the compiler from fusing or
// reassociating these steps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // needs |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = df_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_fast_two_sum(p, e);
}

// 1/d as a double-float: r = rn(1/d); the residual 1 - d r is exact in one
// fma, and r (1 + residual) carries the quotient to about 2^-46.
__device__ __forceinline__ df df_rcp(float d) {
  float r = __frcp_rn(d);
  float res = __fmaf_rn(-d, r, 1.0f);
  return df_fast_two_sum(r, __fmul_rn(r, res));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ bool df_lt(df a, df b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

__device__ __forceinline__ bool df_pos(df a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }

// (a - b) rounded to float; exact in the hi parts when a and b are close.
__device__ __forceinline__ float df_diff(df a, df b) {
  return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

// |(u, v, w)| in float32 with the products and sums in a fixed order (u^2
// rounded, then two fused multiply-adds), so that every inlined copy of the
// walk, whatever the compiler would otherwise contract, gets the same bits.
__device__ __forceinline__ float norm3(float u, float v, float w) {
  return sqrtf(__fmaf_rn(w, w, __fmaf_rn(v, v, __fmul_rn(u, u))));
}

// floor(a) clamped to [0, n-1].
__device__ __forceinline__ int df_floor_clamp(df a, int n) {
  float f = floorf(a.hi);
  if (f == a.hi && a.lo < 0.f) f -= 1.f;
  f = fminf(fmaxf(f, 0.f), (float)(n - 1));
  return (int)f;
}

// ---------------------------------------------------------------------------
// Energy group: half-open [e_g, e_g+1), last group closed (edges in smem).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int group_of(const double *edges, int G, double e) {
  if (edges == nullptr) return 0;
  if (!(e >= edges[0]) || e > edges[G]) return -1;
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (edges[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Cross sections of every material at one energy (Sec. 3: hash-based lookup
// (Brown) on the union log-energy grid, then linear-linear interpolation).
// The hash bin of log2(E) gives a short bracket of grid intervals; a bounded
// fix-up makes the bracket exact whatever the rounding of log2, and a binary
// search inside it finds E[i] <= e < E[i+1].  The interpolation fraction is
// formed in double precision once per ray; the per-material interpolation is
// float32 (the paper's single-precision cross sections).
// Writes sigma to sg[m*stride] and its reciprocal to inv[m*stride].
// ---------------------------------------------------------------------------
// 1/s for s > 0 (0 for s <= 0) in the form's precision: the correctly
// rounded float32 reciprocal, or the float64 one from m64::rcp.
template <typename InvT>
__device__ __forceinline__ InvT recip(float s);
template <>
__device__ __forceinline__ float recip<float>(float s) { return s > 0.f ? __frcp_rn(s) : 0.f; }
template <>
__device__ __forceinline__ double recip<double>(float s) { return s > 0.f ? m64::rcp(s) : 0.0; }

template <typename InvT>
__device__ __forceinline__ void xs_lookup(const XsDev &xs, const int32_t *hash_s, float E,
                                          float *sg, InvT *inv, int stride) {
  const int n = xs.n_union;
  if (n == 0) {
    for (int m = 0; m < xs.n_mat; ++m) { sg[m * stride] = 0.f; inv[m * stride] = InvT(0); }
    return;
  }
  const double e = (double)E;
  int i;
  float f;
  if (n == 1 || e <= __ldg(xs.E)) {
    i = 0; f = 0.f;
  } else if (e >= __ldg(xs.E + n - 1)) {
    i = n - 1; f = 0.f;
  } else {
    int b = (int)((__log2f(E) - xs.l2min) * xs.inv_bw);
    b = min(max(b, 0), xs.n_hash - 1);
    int lo = hash_s[b];
    int hi = min(hash_s[b + 1] + 1, n - 1);
    while (lo > 0 && __ldg(xs.E + lo) > e) --lo;       // fix-up: E[lo] <= e
    while (hi < n - 1 && __ldg(xs.E + hi) <= e) ++hi;  // fix-up: e < E[hi]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (__ldg(xs.E + mid) <= e) lo = mid; else hi = mid;
    }
    i = lo;
    f = (float)((e - __ldg(xs.E + i)) * __ldg(xs.inv_dE + i));
  }
  const float *r0 = xs.S + (int64_t)i * xs.m_pad;
  const float *r1 = (f == 0.f) ? r0 : r0 + xs.m_pad;
  for (int m = 0; m < xs.n_mat; ++m) {
    float a = __ldg(r0 + m), b = __ldg(r1 + m);
    float s = fmaf(f, b - a, a);
    sg[m * stride] = s;
    inv[m * stride] = recip<InvT>(s);
  }
}

// ---------------------------------------------------------------------------
// float -> double without the FP64 pipe (GB300's FP64 rate is 1/64 of FP32):
// a normal float's sign, exponent (rebiased by 1023 - 127 = 896) and
// mantissa are moved into the double's fields with integer operations.
// Zero maps to +0; subnormal inputs (rare: a score below 1.2e-38) take the
// hardware conversion.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u) return (b & 0x7fffffffu) ? (double)f : 0.0;
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// ---------------------------------------------------------------------------
// Eq. 4 along one ray, in the two precision forms.  score() returns the
// segment's contribution as a double; an exact +0 (the transmitted fraction
// has underflowed) needs no tally update, since adding +0 changes no bit.
// Once the transmitted fraction T is exactly 0 it stays 0 (the optical depth
// only grows), so every later score of the ray is exactly +0: score() then
// returns at once and the walk goes on only to cross (and count) the cells.
// ---------------------------------------------------------------------------
template <int FORM>
struct Attenuation;

// Plain form: the ray's weight times its transmitted fraction, W = wt
// exp(-tau_in), carried in float64.  The cell's factor e^-x, x = Sigma l, and
// the path term's e^-x - 1 both come from one float64 range reduction
// (vrc_math64.h: within 0.6 and 2 ulp of the exact values), indexed from the
// float32 product Sigma l.  A void cell (Sigma = 0) has x = 0, factor exactly
// 1 and path term l.  The float32 inputs are widened, their exact product x
// is formed and W is tested for zero with integer operations, which leaves
// the FP64 pipe to the 13 float64 arithmetic operations of a segment.  A segment's (e^-x, path term) needs
// no ray state (terms); the score and the carry W *= e^-x do (apply), so the
// warp-batched walk can compute the first for any lane's segment.  score()
// returns the float64 contribution.
template <>
struct Attenuation<kFormPlain> {
  typedef double inv_t;
  typedef double score_t;
  double T;  // wt exp(-tau) at the entry of the current cell (never -0)
  __device__ __forceinline__ explicit Attenuation(float w) : T(f2d_bits(w)) {}
  __device__ __forceinline__ bool dead() const { return __double_as_longlong(T) == 0; }
  // (e^-x, path term): path term = -(e^-x - 1)/Sigma, or l in void
  __device__ __forceinline__ static double2 terms(float sig, double inv, float l) {
    const double ld = f2d_bits(l);
    const double x = m64::exact_product(sig, l);
    double factor, em;
    m64::exp_expm1(-x, -(sig * l), &factor, &em);
    return make_double2(factor, sig > 0.f ? -em * inv : ld);
  }
  // Score W * path term, then W *= e^-x (W = 0: score 0, nothing changes).
  __device__ __forceinline__ double apply(double2 fp) {
    if (dead()) return 0.0;
    const double s = T * fp.y;
    T *= fp.x;
    return s;
  }
  __device__ __forceinline__ double score(float sig, double inv, float l) {
    if (dead()) return 0.0;
    return apply(terms(sig, inv, l));
  }
  __device__ __forceinline__ static double to_double(double s) { return s; }
};

// FP32 form: optical depth as a compensated float32 pair, exponentials in
// float32; only the tally accumulation stays float64.  One exponential per
// segment: T = exp(-tau) at the cell exit is recomputed from the compensated
// optical depth and carried as the next cell's entry value.  The path term
// (1 - e^-x)/Sigma, x = Sigma l, is (T_in - T_out)/Sigma for x >= 1/8 (the
// difference of two transmitted fractions within a few ulp loses at most a
// factor 1/x = 8 of relative accuracy) and l (1 - e^-x)/x from the Taylor
// series sum_k (-x)^k/(k+1)! to k = 6 below (truncation < 6e-11 at x = 1/8).
// Both are formed and one is selected, so lanes do not diverge on x.
template <>
struct Attenuation<kFormFp32> {
  typedef float inv_t;
  typedef float score_t;
  df tau = {0.f, 0.f};
  float T = 1.f;  // exp(-tau) at the entry of the current cell
  float wt;
  __device__ __forceinline__ explicit Attenuation(float w) : wt(w) {}
  __device__ __forceinline__ float score(float sig, float inv, float l) {
    if (T == 0.f) return 0.f;
    if (!(sig > 0.f)) return wt * T * l;  // void: T unchanged
    const float x = sig * l;
    tau = df_add_f(tau, x);
    const float T_out = expf(-tau.hi) * (1.0f - tau.lo);
    float q = -1.f / 5040.f;
    q = fmaf(q, x, 1.f / 720.f);
    q = fmaf(q, x, -1.f / 120.f);
    q = fmaf(q, x, 1.f / 24.f);
    q = fmaf(q, x, -1.f / 6.f);
    q = fmaf(q, x, 0.5f);
    q = fmaf(q, -x, 1.f);
    const float a = x < 0.125f ? T * (l * q) : (T - T_out) * inv;
    T = T_out;
    return wt * a;
  }
  __device__ __forceinline__ bool dead() const { return T == 0.f; }
  __device__ __forceinline__ static double to_double(float s) { return f2d_bits(s); }
};

// ---------------------------------------------------------------------------
// Score sinks: where the walk puts each segment's score.
// ---------------------------------------------------------------------------
// The tally: one float64 reduction (fire-and-forget red) into the ray's
// group slice, with an L2 evict-last cache policy.  One group's slice of a
// large tally (128 MiB at 256^3) is about the size of the L2; the hint keeps
// tally lines resident ahead of the streamed ray records (measured 5 % less
// time at 256^3 x 16 groups).
struct TallySink {
  double *tal;
  uint64_t policy;  // L2 evict-last access policy, created once per ray
  __device__ __forceinline__ void add(int cell, double v) const {
    asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.f64 [%0], %1, %2;"
                 :: "l"(tal + cell), "d"(v), "l"(policy) : "memory");
  }
};

// Per-history cast: each score goes out as one (key, value) pair with a plain
// store into the ray's own stretch of the pair buffer (nothing to wait
// for); the pairs are summed per (history, bin) after the cast.  The sink
// also counts the pairs of each bucket of 2^bshift consecutive bins for the
// bucket sort that follows, with one fire-and-forget reduction per run of
// the ray's pairs in one bucket.  A ray that would write more pairs than
// its room (an upper bound of its segments) sets kStatusTableFull and drops
// the rest.  The bucket table, shift and status come from the cast's
// arguments (kernel parameters), not from registers.
struct PairSink {
  ulonglong2 *out;            // this ray's stretch
  unsigned long long kbase;   // (group * ncells) << 32 | history id
  uint32_t cap;
  const CastArgs &a;
  mutable uint32_t n, bcur, brun;  // pairs written; the current bucket run
  __device__ __forceinline__ void add(int cell, double v) const {
    if (n < cap) {
      out[n] = make_ulonglong2(kbase + ((unsigned long long)(unsigned)cell << 32),
                               (unsigned long long)__double_as_longlong(v));
      const uint32_t b = ((uint32_t)(kbase >> 32) + (uint32_t)cell) >> a.pout.bshift;
      if (b != bcur) {
        if (brun) atomicAdd(a.pout.bcount + bcur, brun);
        bcur = b;
        brun = 0;
      }
      ++brun;
    } else {
      atomicOr(a.status, kStatusTableFull);
    }
    ++n;
  }
};

// Sink of ray r in group g for a plain cast and for a per-history cast, and
// what a ray leaves behind when its walk ends.
struct TallyMaker {
  __device__ __forceinline__ static TallySink make(const CastArgs &a, int64_t, int g) {
    uint64_t policy;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
    return {a.tally + (int64_t)g * a.mesh.ncells, policy};
  }
  __device__ __forceinline__ static void finish(const CastArgs &, int64_t, const TallySink &) {}
};
struct PairMaker {
  __device__ __forceinline__ static PairSink make(const CastArgs &a, int64_t r, int g) {
    return {a.pout.pairs + pair_off(a.pout, r),
            (((unsigned long long)g * (unsigned long long)a.mesh.ncells) << 32) | __ldg(a.hist + r),
            pair_cap(a.pout, r), a, 0u, 0xffffffffu, 0u};
  }
  __device__ __forceinline__ static void finish(const CastArgs &a, int64_t r, const PairSink &s) {
    a.pout.cnt[r] = s.n < s.cap ? s.n : s.cap;
    if (s.brun) atomicAdd(a.pout.bcount + s.bcur, s.brun);
  }
};

// The walk of one ray through a uniform mesh, one cell per step.  The ray
// is the half-line p + s d, s >= 0, with d not necessarily unit: crossing
// parameters are in units of |d| and lengths are scaled by |d| at the end.
// The crossing parameter of plane j on axis k, ((org_k - p_k) + j h_k) *
// (1/d_k), is evaluated in double-float; the sum is formed before the
// product, so a start exactly on a plane gives an exactly zero first segment,
// as in exact arithmetic.  A start outside the box is clipped to it (vacuum
// outside).  Per axis: S0 = first crossing ahead of the start; B = h |1/d|,
// the spacing of later crossings, which are S0 + m B after m steps on that
// axis (a sum of two positive terms: about 2^-46 relative, no
// cancellation); cnt = planes that axis crosses before the ray leaves the
// mesh.
struct UniformWalk {
  df S[3], S0[3], B[3];
  float m[3], cnt[3];
  int cst[3];
  int cell;
  unsigned mat;  // material of `cell`
  df s_cur;      // crossing parameter of the current cell's entry

  // The nearest crossing ahead: the segment's exit and the next cell.
  struct Next {
    df Sk;
    int k;
    float mk;
    bool leaving;  // the crossing is the mesh boundary
    int ncell;
  };

  // Sets up the walk; false if the ray misses the mesh (dn is not used).
  __device__ __forceinline__ bool init(const MeshDev &M, float px, float py, float pz, float u,
                                       float v, float w, float = 0.f) {
    const float p[3] = {px, py, pz};
    const float d[3] = {u, v, w};
    const df inf = {INFINITY, 0.f};
    df D[3], R[3];  // org - p and 1/d per axis
    df s_in = {0.f, 0.f}, s_out = inf;
    bool miss = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      D[k] = df_add_f(M.org[k], -p[k]);
      const df Dn = df_add(D[k], df_mul_f(M.h[k], (float)M.n[k]));
      if (d[k] == 0.f) {
        R[k] = {0.f, 0.f};
        if (df_pos(D[k]) || !df_pos(Dn)) miss = true;  // p < lo or p >= hi
      } else {
        R[k] = df_rcp(d[k]);
        df a = df_mul(D[k], R[k]);
        df b = df_mul(Dn, R[k]);
        if (d[k] < 0.f) { df t = a; a = b; b = t; }
        if (df_lt(s_in, a)) s_in = a;
        if (df_lt(b, s_out)) s_out = b;
      }
    }
    if (miss || !df_lt(s_in, s_out)) return false;

    cell = 0;
    const int cstride[3] = {1, M.n[0], M.n[0] * M.n[1]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      df c = df_add_f(df_neg(M.org[k]), p[k]);  // p - org
      if (s_in.hi > 0.f && d[k] != 0.f) c = df_add(c, df_mul_f(s_in, d[k]));
      const int ik = df_floor_clamp(df_mul(c, M.inv_h[k]), M.n[k]);
      cell += ik * cstride[k];
      m[k] = 0.f;
      if (d[k] == 0.f) {
        S[k] = inf; S0[k] = inf; B[k] = {0.f, 0.f}; cnt[k] = -1.f; cst[k] = 0;
      } else {
        const bool fwd = d[k] > 0.f;
        S0[k] = df_mul(df_add(D[k], df_mul_f(M.h[k], (float)(ik + (fwd ? 1 : 0)))), R[k]);
        B[k] = df_mul(M.h[k], fwd ? R[k] : df_neg(R[k]));
        S[k] = S0[k];
        cnt[k] = (float)(fwd ? M.n[k] - 1 - ik : ik);
        cst[k] = fwd ? cstride[k] : -cstride[k];
      }
    }
    s_cur = s_in;
    mat = __ldg(M.mat + cell);
    return true;
  }

  // Axis of the nearest crossing (ties resolved x, then y, then z).
  __device__ __forceinline__ Next next() const {
    Next t;
    const bool y_first = df_lt(S[1], S[0]);
    t.Sk = y_first ? S[1] : S[0];
    const bool z_first = df_lt(S[2], t.Sk);
    if (z_first) t.Sk = S[2];
    t.k = z_first ? 2 : (y_first ? 1 : 0);
    t.mk = t.k == 0 ? m[0] : t.k == 1 ? m[1] : m[2];
    t.leaving = t.mk == (t.k == 0 ? cnt[0] : t.k == 1 ? cnt[1] : cnt[2]);
    t.ncell = cell + (t.k == 0 ? cst[0] : t.k == 1 ? cst[1] : cst[2]);
    return t;
  }

  // Length of the current cell's segment, ending at crossing t.
  __device__ __forceinline__ float length(const Next &t, float dn) const {
    return fmaxf(df_diff(t.Sk, s_cur), 0.f) * dn;
  }

  // Steps into t's cell, whose material is nmat.
  __device__ __forceinline__ void advance(const MeshDev &, const Next &t, unsigned nmat) {
    s_cur = t.Sk;
    cell = t.ncell;
    mat = nmat;
    const float mn = t.mk + 1.f;
    const df Sn = df_add(t.k == 0 ? S0[0] : t.k == 1 ? S0[1] : S0[2],
                         df_mul_f(t.k == 0 ? B[0] : t.k == 1 ? B[1] : B[2], mn));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == t.k) { m[a] = mn; S[a] = Sn; }
    }
  }
};

// Steps of the walk per loop iteration, by score sink.
template <typename Sink>
constexpr int kWalkUnroll = 2;
template <>
constexpr int kWalkUnroll<PairSink> = 1;

// Walks one ray through the mesh (Walk: UniformWalk or RectWalk) and adds
// its Eq. 4 score to every crossed cell through `sink` (the ray's group
// slice of the tally, or its history's slots).  The walk ends when the ray
// leaves the mesh or after max_steps steps (then *overflow is set).  Returns
// the number of positive-length segments walked; nlive counts the scores
// added to the sink.
template <int FORM, typename Walk, typename Sink>
__device__ __forceinline__ uint32_t cast_ray_walk(const MeshDev &M, float px, float py, float pz,
                                                  float u, float v, float w, float wt, float dn,
                                                  const Sink &sink, const float *sg,
                                                  const typename Attenuation<FORM>::inv_t *inv,
                                                  int stride, bool stop_zero, bool *overflow,
                                                  uint32_t &nlive) {
  Walk W;
  if (!W.init(M, px, py, pz, u, v, w, dn)) return 0;
  Attenuation<FORM> att(wt);
  uint32_t nseg = 0;
  const int max_steps = M.n[0] + M.n[1] + M.n[2] + 3;
  // two steps per loop iteration with a tally sink: FP32 cast 2.8 % faster
  // on slab256 (four: 1.4 %, with more spills), 2.2 % on the graded mesh;
  // the per-history pair sink runs 1.4 % slower unrolled and is not
#pragma unroll(kWalkUnroll<Sink>)
  for (int step = 0;; ++step) {
    if (stop_zero && att.dead()) break;  // every later score is +0 (opt-in)
    const typename Walk::Next t = W.next();
    // FP32 form: once every score is +0 the walk skips the loads of the next
    // cell's material and of sigma (the plain form measured faster keeping them)
    const bool live = FORM == kFormFp32 ? !att.dead() : true;
    const unsigned nmat = (t.leaving || !live) ? 0u : __ldg(M.mat + t.ncell);  // prefetch the next cell

    const float l = W.length(t, dn);
    if (live) {
      typename Attenuation<FORM>::score_t sc;
      if constexpr (FORM == kFormFp32) {  // sigma and 1/sigma interleaved: one 8-byte load
        const float2 si = *reinterpret_cast<const float2 *>(sg + W.mat * stride);
        sc = att.score(si.x, si.y, l);
      } else {
        sc = att.score(sg[W.mat * stride], inv[W.mat * stride], l);
      }
      if (sc != 0) {
        sink.add(W.cell, Attenuation<FORM>::to_double(sc));
        ++nlive;
      }
    }
    nseg += l > 0.f;

    if (t.leaving) break;
    if (step >= max_steps) { *overflow = true; break; }
    W.advance(M, t, nmat);
  }
  return nseg;
}

// Plane j on axis k of a rectilinear mesh.
__device__ __forceinline__ df mesh_plane(const MeshDev &M, int k, int j) {
  const float2 e = __ldg(M.edge[k] + j);
  return {e.x, e.y};
}

// Cell index on axis k of a rectilinear mesh holding coordinate c:
// edge[j] <= c < edge[j+1] by binary search, clamped to 0..n-1.
__device__ __forceinline__ int locate_rect(const MeshDev &M, int k, df c) {
  const int n = M.n[k];
  if (!df_lt(c, mesh_plane(M, k, n))) return n - 1;
  if (df_lt(c, mesh_plane(M, k, 0))) return 0;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (df_lt(c, mesh_plane(M, k, mid))) hi = mid; else lo = mid;
  }
  return lo;
}

// The walk of one ray through a rectilinear mesh (planes at given positions
// per axis).  The crossing of plane j on axis k, (edge_k[j] - p_k) * (1/d_k),
// is evaluated in double-float from the plane index at every step (never
// accumulated); the walk leaves the mesh when the stepped axis crosses its
// last plane.  Per axis: J = index of the next plane ahead, last = the plane
// that leaves the mesh, js = +-1 plane step.
struct RectWalk {
  float p[3];
  df R[3];  // 1/d per axis
  df S[3];
  int J[3], last[3], js[3], cst[3];
  int cell;
  unsigned mat;  // material of `cell`
  df s_cur;      // crossing parameter of the current cell's entry

  struct Next {
    df Sk;
    int k;
    int Jk;
    bool leaving;  // the crossing is the mesh boundary
    int ncell;
  };

  // Sets up the walk; false if the ray misses the mesh (dn is not used).
  __device__ __forceinline__ bool init(const MeshDev &M, float px, float py, float pz, float u,
                                       float v, float w, float = 0.f) {
    p[0] = px; p[1] = py; p[2] = pz;
    const float d[3] = {u, v, w};
    const df inf = {INFINITY, 0.f};
    df s_in = {0.f, 0.f}, s_out = inf;
    bool miss = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const df D0 = df_add_f(mesh_plane(M, k, 0), -p[k]);
      const df Dn = df_add_f(mesh_plane(M, k, M.n[k]), -p[k]);
      if (d[k] == 0.f) {
        R[k] = {0.f, 0.f};
        if (df_pos(D0) || !df_pos(Dn)) miss = true;  // p < lo or p >= hi
      } else {
        R[k] = df_rcp(d[k]);
        df a = df_mul(D0, R[k]);
        df b = df_mul(Dn, R[k]);
        if (d[k] < 0.f) { df t = a; a = b; b = t; }
        if (df_lt(s_in, a)) s_in = a;
        if (df_lt(b, s_out)) s_out = b;
      }
    }
    if (miss || !df_lt(s_in, s_out)) return false;

    cell = 0;
    const int cstride[3] = {1, M.n[0], M.n[0] * M.n[1]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      df c = {p[k], 0.f};
      if (s_in.hi > 0.f && d[k] != 0.f) c = df_add(c, df_mul_f(s_in, d[k]));
      const int ik = locate_rect(M, k, c);
      cell += ik * cstride[k];
      if (d[k] == 0.f) {
        S[k] = inf; J[k] = 0; last[k] = -1; js[k] = 0; cst[k] = 0;
      } else {
        const bool fwd = d[k] > 0.f;
        J[k] = fwd ? ik + 1 : ik;
        last[k] = fwd ? M.n[k] : 0;
        js[k] = fwd ? 1 : -1;
        cst[k] = fwd ? cstride[k] : -cstride[k];
        S[k] = df_mul(df_add_f(mesh_plane(M, k, J[k]), -p[k]), R[k]);
      }
    }
    s_cur = s_in;
    mat = __ldg(M.mat + cell);
    return true;
  }

  // Axis of the nearest crossing (ties resolved x, then y, then z).
  __device__ __forceinline__ Next next() const {
    Next t;
    const bool y_first = df_lt(S[1], S[0]);
    t.Sk = y_first ? S[1] : S[0];
    const bool z_first = df_lt(S[2], t.Sk);
    if (z_first) t.Sk = S[2];
    t.k = z_first ? 2 : (y_first ? 1 : 0);
    t.Jk = t.k == 0 ? J[0] : t.k == 1 ? J[1] : J[2];
    t.leaving = t.Jk == (t.k == 0 ? last[0] : t.k == 1 ? last[1] : last[2]);
    t.ncell = cell + (t.k == 0 ? cst[0] : t.k == 1 ? cst[1] : cst[2]);
    return t;
  }

  // Length of the current cell's segment, ending at crossing t.
  __device__ __forceinline__ float length(const Next &t, float dn) const {
    return fmaxf(df_diff(t.Sk, s_cur), 0.f) * dn;
  }

  // Steps into t's cell, whose material is nmat.
  __device__ __forceinline__ void advance(const MeshDev &M, const Next &t, unsigned nmat) {
    s_cur = t.Sk;
    cell = t.ncell;
    mat = nmat;
    const int Jn = t.Jk + (t.k == 0 ? js[0] : t.k == 1 ? js[1] : js[2]);
    const float pk = t.k == 0 ? p[0] : t.k == 1 ? p[1] : p[2];
    const df Sn = df_mul(df_add_f(mesh_plane(M, t.k, Jn), -pk),
                         t.k == 0 ? R[0] : t.k == 1 ? R[1] : R[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == t.k) { J[a] = Jn; S[a] = Sn; }
    }
  }
};

// ---------------------------------------------------------------------------
// Plain form, with the float64 work shared by the warp.
// A float64 operation occupies GB300's FP64 pipe for a whole warp however
// few of its lanes are active, and the lanes of a warp reach the ends of
// their rays' live stretches at different steps.  So the walk and the score
// are split: in rounds, every lane walks up to kPlainBatch steps of its ray
// and queues each positive-length segment that can still score (sigma,
// length, 1/sigma, cell) in the warp's shared-memory queue; the warp then
// computes e^-x and the path term (-(e^-x - 1)/Sigma, or l in void) for all
// queued segments, 32 at a time, each lane taking any lane's segment; last,
// each lane applies its own segments in order: score = W * path term, W *=
// e^-x, tally add.  Each score is Attenuation<kFormPlain>::score's,
// operation for operation.  A segment is queued only while the ray's
// float32 optical depth is below 760 + max(0, ln wt): beyond that W = wt
// e^-tau is below 1e-322 (e^-745.2 is below half the smallest subnormal),
// so its scores are 0, or below 1e-322 where rounding holds W at the
// smallest subnormal; they are dropped.  The float32 depth is accurate to
// far better than the margin.  Warp-collective: all 32 lanes call it, `active` false for a
// lane without a ray.  Every lane's walk ends within max_steps + 1 steps, so
// the rounds end.
// ---------------------------------------------------------------------------
constexpr int kPlainBatch = 10;

// A warp's queue: io[32 kPlainBatch] holds (sigma, length, 1/sigma) and then
// (e^-x, path term) per segment, lane-major; cell[32 kPlainBatch]; slot[32
// kPlainBatch] lists the io slots of the round's segments in compacted order.
struct WarpQueue {
  double2 *io;
  int32_t *cell;
  int32_t *slot;
};

// Shared-memory bytes of one warp's queue (16-byte multiple).
constexpr size_t kWarpQueueBytes = 32 * kPlainBatch * (sizeof(double2) + 2 * sizeof(int32_t));

// The calling warp's queue in a block's queue area (kWarpQueueBytes per warp,
// 16-byte aligned).
__device__ __forceinline__ WarpQueue warp_queue(unsigned char *area) {
  unsigned char *q = area + kWarpQueueBytes * (threadIdx.x / 32);
  return {reinterpret_cast<double2 *>(q),
          reinterpret_cast<int32_t *>(q + 32 * kPlainBatch * sizeof(double2)),
          reinterpret_cast<int32_t *>(q + 32 * kPlainBatch * (sizeof(double2) + sizeof(int32_t)))};
}

// One queued segment's (e^-x, path term) from its (sigma, length, 1/sigma).
__device__ __forceinline__ double2 plain_terms(double2 in) {
  return Attenuation<kFormPlain>::terms(__int_as_float(__double2loint(in.x)),
                                        in.y, __int_as_float(__double2hiint(in.x)));
}

template <typename Walk, typename Sink>
__device__ __forceinline__ uint32_t cast_ray_plain_warp(const MeshDev &M, bool active, float px,
                                                        float py, float pz, float u, float v, float w,
                                                        float wt, float dn, const Sink &sink,
                                                        const float *sg, const double *inv,
                                                        int stride, bool stop_zero, bool *overflow,
                                                        const WarpQueue &Q, uint32_t &nlive) {
  const unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  Walk W;
  if (active) active = W.init(M, px, py, pz, u, v, w, dn);
  Attenuation<kFormPlain> att(wt);  // W at the entry of the next segment to apply
  float tau = 0.f;                   // float32 optical depth walked so far
  const float tau_dead = 760.f + (wt > 1.f ? __logf(wt) : 0.f);
  uint32_t nseg = 0;
  const int max_steps = M.n[0] + M.n[1] + M.n[2] + 3;
  int step = 0;
  for (;;) {
    // 1. walk: queue up to kPlainBatch segments of this lane's ray
    int nq = 0;
    if (active && stop_zero && att.dead()) active = false;
    for (int j = 0; j < kPlainBatch && active; ++j) {
      const typename Walk::Next t = W.next();
      const unsigned nmat = t.leaving ? 0u : __ldg(M.mat + t.ncell);  // prefetch the next cell
      const float l = W.length(t, dn);
      if (l > 0.f) {
        ++nseg;
        if (tau < tau_dead) {
          const float sig = sg[W.mat * stride];
          const int slot = lane * kPlainBatch + nq;
          Q.io[slot] = make_double2(__hiloint2double(__float_as_int(l), __float_as_int(sig)),
                                    inv[W.mat * stride]);
          Q.cell[slot] = W.cell;
          ++nq;
          tau = fmaf(sig, l, tau);
        }
      }
      if (t.leaving) { active = false; break; }
      if (step >= max_steps) { *overflow = true; active = false; break; }
      ++step;
      W.advance(M, t, nmat);
    }
    // 2. e^-x and path terms of every queued segment, 32 at a time
    __syncwarp(kAll);
    int incl = nq;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kAll, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(kAll, incl, 31);
    for (int j = 0; j < nq; ++j) Q.slot[incl - nq + j] = lane * kPlainBatch + j;
    __syncwarp(kAll);
    for (int gi = lane; gi < total; gi += 32) {
      const int slot = Q.slot[gi];
      Q.io[slot] = plain_terms(Q.io[slot]);
    }
    __syncwarp(kAll);
    // 3. this lane's scores, in walk order
    for (int j = 0; j < nq; ++j) {
      const int slot = lane * kPlainBatch + j;
      const double sc = att.apply(Q.io[slot]);
      if (sc != 0.0) {
        sink.add(Q.cell[slot], sc);
        ++nlive;
      }
    }
    if (!__any_sync(kAll, active)) break;
  }
  return nseg;
}

// The eight fields of ray r (SoA or 32-byte records).
__device__ __forceinline__ void load_ray(const RayPtrs &R, int64_t r, float (&f)[8]) {
  if (R.aos) {
    const float4 a = __ldg(R.aos + 2 * r), b = __ldg(R.aos + 2 * r + 1);
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
    f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
  } else {
    f[0] = __ldg(R.x + r); f[1] = __ldg(R.y + r); f[2] = __ldg(R.z + r); f[3] = __ldg(R.u + r);
    f[4] = __ldg(R.v + r); f[5] = __ldg(R.w + r); f[6] = __ldg(R.E + r); f[7] = __ldg(R.wt + r);
  }
}

// Per-thread counters of one cast, flushed with one atomic per warp.
struct RayCounts {
  uint32_t seg = 0, rays = 0, rej = 0, ovf = 0, live = 0;
};

// A validated ray: position, direction (and its norm), weight, group.
struct RayIn {
  float x, y, z, u, v, w, wt, dn;
  int g;
};

// Loads ray r, validates it, finds its group and writes the cross sections
// of every material at its energy (and their reciprocals) to this thread's
// columns of sig_s / inv_s.  False for a rejected ray (counted) or one
// outside the group structure.
template <int FORM, bool SURR>
__device__ __forceinline__ bool ray_setup(const CastArgs &a, int64_t r, const int32_t *hash_s,
                                          const double *edges, float *sig_s,
                                          typename Attenuation<FORM>::inv_t *inv_s, int stride,
                                          RayCounts &c, RayIn &ray) {
  float f[8];
  load_ray(a.rays, r, f);
  const float x = f[0], y = f[1], z = f[2], u = f[3], v = f[4], w = f[5], E = f[6], wt = f[7];
  ++c.rays;
  const float dn = norm3(u, v, w);
  if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(u) && isfinite(v) && isfinite(w) &&
        isfinite(E) && isfinite(wt) && E > 0.f && dn > 0.f && isfinite(dn))) {
    ++c.rej;
    return false;
  }
  const int g = group_of(edges, a.n_groups, (double)E);
  if (g < 0) return false;
  bool from_table = true;
  if (SURR) {  // surrogate sigma for the leading rays (those in accepted energy bins)
    if (r < (int64_t)__ldg(a.n_surr)) {
      const float4 *q = reinterpret_cast<const float4 *>(a.sig_ray + r * 16);
      from_table = false;
      for (int m4 = 0; m4 < (a.xs.n_mat + 3) / 4; ++m4) {
        const float4 v = __ldg(q + m4);
        const float s4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int m = 4 * m4 + e;
          if (m < a.xs.n_mat) {
            sig_s[m * stride] = s4[e];
            inv_s[m * stride] = recip<typename Attenuation<FORM>::inv_t>(s4[e]);
          }
        }
      }
    }
  }
  if (from_table) xs_lookup(a.xs, hash_s, E, sig_s, inv_s, stride);
  ray = {x, y, z, u, v, w, wt, dn, g};
  return true;
}

// One ray of a cast: validation, group, cross sections, walk and score.
template <int FORM, bool SURR = false, typename Maker = TallyMaker, bool RECT = false>
__device__ __forceinline__ void cast_one(const CastArgs &a, int64_t r, const int32_t *hash_s,
                                         const double *edges, float *sig_s,
                                         typename Attenuation<FORM>::inv_t *inv_s, int stride,
                                         RayCounts &c) {
  RayIn q;
  if (!ray_setup<FORM, SURR>(a, r, hash_s, edges, sig_s, inv_s, stride, c, q)) return;
  bool ovf = false;
  typedef typename std::conditional<RECT, RectWalk, UniformWalk>::type Walk;
  const auto sink = Maker::make(a, r, q.g);
  c.seg += cast_ray_walk<FORM, Walk>(a.mesh, q.x, q.y, q.z, q.u, q.v, q.w, q.wt, q.dn, sink, sig_s,
                                     inv_s, stride, a.stop_zero != 0, &ovf, c.live);
  Maker::finish(a, r, sink);
  c.ovf += ovf;
}

// One ray per lane of a warp, plain form, through the warp-batched walk
// (cast_ray_plain_warp) on a uniform or rectilinear mesh.  Warp-collective:
// every lane calls it, with has_ray false where its index is past the last
// ray.
template <bool SURR, typename Maker, bool RECT>
__device__ __forceinline__ void cast_one_plain_warp(const CastArgs &a, int64_t r, bool has_ray,
                                                    const int32_t *hash_s, const double *edges,
                                                    float *sig_s, double *inv_s, int stride,
                                                    const WarpQueue &Q, RayCounts &c) {
  typedef typename std::conditional<RECT, RectWalk, UniformWalk>::type Walk;
  RayIn q = {};
  const bool ok =
      has_ray && ray_setup<kFormPlain, SURR>(a, r, hash_s, edges, sig_s, inv_s, stride, c, q);
  bool ovf = false;
  // a lane without a ray builds its (unused) sink from ray 0 of group 0
  const auto sink = Maker::make(a, ok ? r : 0, ok ? q.g : 0);
  c.seg += cast_ray_plain_warp<Walk>(a.mesh, ok, q.x, q.y, q.z, q.u, q.v, q.w, q.wt, q.dn, sink, sig_s,
                                     inv_s, stride, a.stop_zero != 0, &ovf, Q, c.live);
  if (ok) Maker::finish(a, r, sink);
  c.ovf += ovf;
}

// Adds a warp's counters to the device counters (all 32 lanes must call).
__device__ __forceinline__ void flush_counts(RayCounts c, unsigned long long *counters,
                                             unsigned int *status) {
  for (int o = 16; o > 0; o >>= 1) {
    c.seg += __shfl_down_sync(0xffffffffu, c.seg, o);
    c.rays += __shfl_down_sync(0xffffffffu, c.rays, o);
    c.rej += __shfl_down_sync(0xffffffffu, c.rej, o);
    c.ovf += __shfl_down_sync(0xffffffffu, c.ovf, o);
    c.live += __shfl_down_sync(0xffffffffu, c.live, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c.seg) atomicAdd(counters + kCntSegments, (unsigned long long)c.seg);
    if (c.rays) atomicAdd(counters + kCntRays, (unsigned long long)c.rays);
    if (c.live) atomicAdd(counters + kCntLive, (unsigned long long)c.live);
    if (c.rej) {
      atomicAdd(counters + kCntRejected, (unsigned long long)c.rej);
      atomicOr(status, kStatusNonfinite);
    }
    if (c.ovf) {
      atomicAdd(counters + kCntOverflow, (unsigned long long)c.ovf);
      atomicOr(status, kStatusTraversal);
    }
  }
}

// Optical depth along the segment p -> q (vacuum outside the mesh) for the
// next-event estimator: the same double-float grid walk as cast_ray, with the
// segment parametrised as p + s (q - p), s in [0, 1], and the last cell cut at
// s = 1.  sg[mat * stride] holds sigma of each material for the ray's energy.
// The walk stops early once tau.hi exceeds tau_zero, a depth at which the
// caller's exp(-tau) is exactly 0 (tau only grows, so the result is the same).
// Returns tau as a compensated float32 pair.
__device__ __forceinline__ df optical_depth(const MeshDev &M, const float p[3], const float q[3],
                                            const float *sg, int stride, float tau_zero,
                                            bool *overflow) {
  const float d[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
  const float dn = norm3(d[0], d[1], d[2]);
  const df inf = {INFINITY, 0.f};
  df tau = {0.f, 0.f};
  df D[3], R[3];
  df s_in = {0.f, 0.f}, s_out = {1.f, 0.f};
  bool miss = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    D[k] = df_add_f(M.org[k], -p[k]);
    const df Dn = df_add(D[k], df_mul_f(M.h[k], (float)M.n[k]));
    if (d[k] == 0.f) {
      R[k] = {0.f, 0.f};
      if (df_pos(D[k]) || !df_pos(Dn)) miss = true;
    } else {
      R[k] = df_rcp(d[k]);
      df a = df_mul(D[k], R[k]);
      df b = df_mul(Dn, R[k]);
      if (d[k] < 0.f) { df t = a; a = b; b = t; }
      if (df_lt(s_in, a)) s_in = a;
      if (df_lt(b, s_out)) s_out = b;
    }
  }
  if (miss || !df_lt(s_in, s_out)) return tau;
  df S[3], S0[3], B[3];
  float m[3];
  int cst[3];
  int cell = 0;
  const int cstride[3] = {1, M.n[0], M.n[0] * M.n[1]};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    df c = df_add_f(df_neg(M.org[k]), p[k]);
    if (s_in.hi > 0.f && d[k] != 0.f) c = df_add(c, df_mul_f(s_in, d[k]));
    const int ik = df_floor_clamp(df_mul(c, M.inv_h[k]), M.n[k]);
    cell += ik * cstride[k];
    m[k] = 0.f;
    if (d[k] == 0.f) {
      S[k] = inf; S0[k] = inf; B[k] = {0.f, 0.f}; cst[k] = 0;
    } else {
      const bool fwd = d[k] > 0.f;
      S0[k] = df_mul(df_add(D[k], df_mul_f(M.h[k], (float)(ik + (fwd ? 1 : 0)))), R[k]);
      B[k] = df_mul(M.h[k], fwd ? R[k] : df_neg(R[k]));
      S[k] = S0[k];
      cst[k] = fwd ? cstride[k] : -cstride[k];
    }
  }
  df s_cur = s_in;
  const int max_steps = M.n[0] + M.n[1] + M.n[2] + 3;
  for (int step = 0;; ++step) {
    const bool y_first = df_lt(S[1], S[0]);
    df Sk = y_first ? S[1] : S[0];
    const bool z_first = df_lt(S[2], Sk);
    if (z_first) Sk = S[2];
    const int k = z_first ? 2 : (y_first ? 1 : 0);
    const bool last = !df_lt(Sk, s_out);  // the segment ends (detector or mesh exit) in this cell
    const df s_end = last ? s_out : Sk;
    const float l = fmaxf(df_diff(s_end, s_cur), 0.f) * dn;
    const float sig = sg[__ldg(M.mat + cell) * stride];
    tau = df_add_f(tau, sig * l);
    if (last || tau.hi > tau_zero) break;
    if (step >= max_steps) { *overflow = true; break; }
    s_cur = Sk;
    cell += k == 0 ? cst[0] : k == 1 ? cst[1] : cst[2];
    const float mn = (k == 0 ? m[0] : k == 1 ? m[1] : m[2]) + 1.f;
    const df Sn = df_add(k == 0 ? S0[0] : k == 1 ? S0[1] : S0[2],
                         df_mul_f(k == 0 ? B[0] : k == 1 ? B[1] : B[2], mn));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == k) { m[a] = mn; S[a] = Sn; }
    }
  }
  return tau;
}

}  // namespace vrc
