/*
 * FP64 CPU oracle for the volumetric-ray-casting (VRC) fluence estimator
 * (Sweezy, "A Monte Carlo Volumetric-Ray-Casting Estimator for Global
 * Fluence Tallies on GPUs", arXiv:1706.07476).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (all in double precision):
 *  - sigma_t(E) per material by binary search on the material's own energy
 *    grid and linear-linear interpolation between table points (Sec. 3:
 *    tabulated continuous-energy data, linearly interpolated), clamped to
 *    the end values outside the table; a material with no table is void
 *    (sigma_t = 0).
 *  - the energy group of a ray: half-open [e_g, e_g+1), last group closed;
 *    rays outside every group score nothing.
 *  - the cells a ray crosses and its length in each, by a 3-D Amanatides-Woo
 *    grid walk on a uniform mesh (planes at x0 + j dx) or a rectilinear one
 *    (planes at given per-axis edges: the non-uniform Cartesian meshes of
 *    the paper's outlook, Sec. 6).  The next crossing on every axis is recomputed from the
 *    integer cell index each step (never accumulated).  The ray is a
 *    half-line from its start point; a start outside the mesh is clipped to
 *    the mesh box (vacuum outside, Sec. 5.1: vacuum boundary only), and the
 *    walk ends when the ray leaves the mesh (Sec. 3: the ray is cast through
 *    the entire geometry).
 *  - the score of Eq. 4 in every crossed cell:
 *        s_i = wt * exp(-tau_in) * (1 - exp(-sigma_i l_i)) / sigma_i
 *    with tau_in the optical depth from the start point to the entry of
 *    cell i (the integral of Eq. 2), evaluated as -expm1(-sigma l)/sigma,
 *    and s_i = wt * exp(-tau_in) * l_i in void (the sigma -> 0 limit).
 *    wt is the per-ray weight W/N of Eq. 4.
 *  - the tally: the sum of s_i over all rays, per (group, cell), layout
 *    [group][iz][iy][ix].
 *
 * A second, independent traversal (orc_trace_brute) collects every plane
 * crossing, sorts them and classifies each interval's midpoint; the tests
 * use it to check the grid walk.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
  int32_t nx, ny, nz;
  double x0, y0, z0, dx, dy, dz;
  const uint8_t *material; /* [nz][ny][nx] */
  /* Optional plane positions per axis (n+1 strictly ascending values each);
   * NULL on every axis = the uniform mesh x0 + j dx.  When set, x0..dz are
   * ignored. */
  const double *xe, *ye, *ze;
} orc_mesh;

/* Concatenated per-material tables: material m owns entries offs[m] ..
 * offs[m+1]-1 of E and S; an empty range is a void material. */
typedef struct {
  int32_t n_materials;
  const double *E;
  const double *S;
  const int64_t *offs;
} orc_xs;

/* ------------------------------------------------------------------ */
/* cross sections and groups                                            */
/* ------------------------------------------------------------------ */

/* sigma_t(e) for one table: binary search for E[i] <= e < E[i+1], then
 * linear-linear interpolation; clamped to S[0] / S[n-1] outside. */
double orc_sigma_t(const double *E, const double *S, int64_t n, double e) {
  if (n <= 0) return 0.0;
  if (n == 1 || e <= E[0]) return S[0];
  if (e >= E[n - 1]) return S[n - 1];
  int64_t lo = 0, hi = n - 1; /* invariant: E[lo] <= e < E[hi] */
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (E[mid] <= e) lo = mid; else hi = mid;
  }
  return S[lo] + (e - E[lo]) * (S[hi] - S[lo]) / (E[hi] - E[lo]);
}

/* group index of energy e; -1 when outside all groups.  edges == NULL or
 * n_groups <= 0 means a single group that takes every energy. */
int32_t orc_group(const double *edges, int32_t n_groups, double e) {
  if (edges == NULL || n_groups <= 0) return 0;
  if (!(e >= edges[0]) || e > edges[n_groups]) return -1;
  if (e == edges[n_groups]) return n_groups - 1;
  int32_t lo = 0, hi = n_groups; /* edges[lo] <= e < edges[hi] */
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) / 2;
    if (edges[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

/* ------------------------------------------------------------------ */
/* traversal                                                            */
/* ------------------------------------------------------------------ */

static const double *axis_edges(const orc_mesh *m, int k) {
  return k == 0 ? m->xe : (k == 1 ? m->ye : m->ze);
}

static int32_t axis_cells(const orc_mesh *m, int k) {
  return k == 0 ? m->nx : (k == 1 ? m->ny : m->nz);
}

/* Position of plane j (0..n) on axis k. */
static double plane(const orc_mesh *m, int k, int64_t j) {
  const double *e = axis_edges(m, k);
  if (e) return e[j];
  const double lo[3] = {m->x0, m->y0, m->z0};
  const double h[3] = {m->dx, m->dy, m->dz};
  return lo[k] + (double)j * h[k];
}

static int32_t clampi(int64_t i, int32_t n) {
  if (i < 0) return 0;
  if (i >= n) return n - 1;
  return (int32_t)i;
}

/* Cell index on axis k of coordinate q: plane(j) <= q < plane(j+1), clamped
 * to 0..n-1. */
static int32_t locate(const orc_mesh *m, int k, double q) {
  const int32_t n = axis_cells(m, k);
  const double *e = axis_edges(m, k);
  if (!e) {
    const double lo[3] = {m->x0, m->y0, m->z0};
    const double h[3] = {m->dx, m->dy, m->dz};
    return clampi((int64_t)floor((q - lo[k]) / h[k]), n);
  }
  if (!(q >= e[0])) return 0;
  if (q >= e[n]) return n - 1;
  int32_t lo = 0, hi = n; /* invariant: e[lo] <= q < e[hi] */
  while (hi - lo > 1) {
    int32_t mid = lo + (hi - lo) / 2;
    if (e[mid] <= q) lo = mid; else hi = mid;
  }
  return lo;
}

/* Clip the half-line p + t d (t >= 0) to the mesh box.  Returns 0 when the
 * ray misses, else 1 with [*t0, *t1] the part inside the box.  On an axis
 * with d == 0 the ray must satisfy lo <= p < hi. */
static int clip_box(const orc_mesh *m, const double p[3], const double d[3], double *t0,
                    double *t1) {
  double a = 0.0, b = INFINITY;
  for (int k = 0; k < 3; ++k) {
    const double lo = plane(m, k, 0);
    const double hi = plane(m, k, axis_cells(m, k));
    if (d[k] == 0.0) {
      if (p[k] < lo || p[k] >= hi) return 0;
      continue;
    }
    double ta = (lo - p[k]) / d[k];
    double tb = (hi - p[k]) / d[k];
    if (ta > tb) { double s = ta; ta = tb; tb = s; }
    if (ta > a) a = ta;
    if (tb < b) b = tb;
  }
  if (!(a < b)) return 0;
  *t0 = a;
  *t1 = b;
  return 1;
}

/* Grid walk.  d must be a unit vector.  Writes, per step, the linear cell
 * index, the entry distance and the length (zero-length steps at exact
 * edge/corner crossings included).  Returns the number of steps, or -1 if
 * more than cap steps would be needed. */
int64_t orc_trace_dda(const orc_mesh *m, const double p[3], const double d[3], int64_t *cells,
                      double *t_in, double *lens, int64_t cap) {
  double t0, t1;
  if (!clip_box(m, p, d, &t0, &t1)) return 0;
  const int32_t n[3] = {m->nx, m->ny, m->nz};
  int32_t idx[3];
  for (int k = 0; k < 3; ++k) idx[k] = locate(m, k, p[k] + t0 * d[k]);
  double t = t0;
  int64_t count = 0;
  for (;;) {
    double tn[3];
    for (int k = 0; k < 3; ++k) {
      if (d[k] > 0.0)
        tn[k] = (plane(m, k, idx[k] + 1) - p[k]) / d[k];
      else if (d[k] < 0.0)
        tn[k] = (plane(m, k, idx[k]) - p[k]) / d[k];
      else
        tn[k] = INFINITY;
    }
    int ks = 0;
    if (tn[1] < tn[ks]) ks = 1;
    if (tn[2] < tn[ks]) ks = 2;
    double l = tn[ks] - t;
    if (l < 0.0) l = 0.0;
    if (count >= cap) return -1;
    cells[count] = ((int64_t)idx[2] * m->ny + idx[1]) * m->nx + idx[0];
    t_in[count] = t;
    lens[count] = l;
    ++count;
    if (tn[ks] > t) t = tn[ks];
    idx[ks] += d[ks] > 0.0 ? 1 : -1;
    if (idx[ks] < 0 || idx[ks] >= n[ks]) break;
  }
  return count;
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Brute-force traversal: every plane crossing x = plane(j) (and y, z)
 * strictly inside the clipped interval is collected and sorted; each
 * positive-length interval's midpoint is classified by locate().  tbuf needs
 * room for nx+ny+nz+5 values.  Returns the number of positive-length
 * segments, or -1 if cap is too small. */
int64_t orc_trace_brute(const orc_mesh *m, const double p[3], const double d[3], int64_t *cells,
                        double *t_in, double *lens, int64_t cap, double *tbuf) {
  double t0, t1;
  if (!clip_box(m, p, d, &t0, &t1)) return 0;
  const int32_t n[3] = {m->nx, m->ny, m->nz};
  int64_t nt = 0;
  tbuf[nt++] = t0;
  tbuf[nt++] = t1;
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0) continue;
    for (int32_t j = 0; j <= n[k]; ++j) {
      double t = (plane(m, k, j) - p[k]) / d[k];
      if (t > t0 && t < t1) tbuf[nt++] = t;
    }
  }
  qsort(tbuf, (size_t)nt, sizeof(double), cmp_double);
  int64_t count = 0;
  for (int64_t i = 0; i + 1 < nt; ++i) {
    double a = tbuf[i], b = tbuf[i + 1];
    if (!(b > a)) continue;
    double mid = 0.5 * (a + b);
    int32_t idx[3];
    for (int k = 0; k < 3; ++k) idx[k] = locate(m, k, p[k] + mid * d[k]);
    if (count >= cap) return -1;
    cells[count] = ((int64_t)idx[2] * m->ny + idx[1]) * m->nx + idx[0];
    t_in[count] = a;
    lens[count] = b - a;
    ++count;
  }
  return count;
}

/* ------------------------------------------------------------------ */
/* scoring                                                              */
/* ------------------------------------------------------------------ */

/* Eq. 4 contribution of one segment with entry optical depth tau. */
static double segment_score(double wt, double tau, double sig, double l) {
  double path = sig > 0.0 ? -expm1(-sig * l) / sig : l;
  return wt * exp(-tau) * path;
}

/* Promote a float32 ray to double and normalise its direction.  Returns 0
 * for a ray that scores nothing: non-finite field, non-positive energy or a
 * zero direction (the caller counts these). */
static int prepare_ray(float x, float y, float z, float u, float v, float w, float E, float wt,
                       double p[3], double d[3]) {
  if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(u) || !isfinite(v) ||
      !isfinite(w) || !isfinite(E) || !isfinite(wt) || !(E > 0.0f))
    return 0;
  p[0] = x; p[1] = y; p[2] = z;
  double norm = sqrt((double)u * u + (double)v * v + (double)w * w);
  if (!(norm > 0.0)) return 0;
  d[0] = u / norm; d[1] = v / norm; d[2] = w / norm;
  return 1;
}

/* Per-segment detail of one ray: cells, entry distance, length, sigma and
 * score (all steps, zero-length ones included).  Returns the step count,
 * 0 for a ray that scores nothing, -1 if cap is too small. */
int64_t orc_ray_segments(const orc_mesh *m, const orc_xs *xs, const double *edges,
                         int32_t n_groups, float x, float y, float z, float u, float v, float w,
                         float E, float wt, int64_t *cells, double *t_in, double *lens,
                         double *sig_out, double *score_out, int64_t cap) {
  double p[3], d[3];
  if (!prepare_ray(x, y, z, u, v, w, E, wt, p, d)) return 0;
  if (orc_group(edges, n_groups, (double)E) < 0) return 0;
  int64_t ns = orc_trace_dda(m, p, d, cells, t_in, lens, cap);
  if (ns <= 0) return ns;
  double tau = 0.0;
  for (int64_t s = 0; s < ns; ++s) {
    int mat = m->material[cells[s]];
    const int64_t a = xs->offs[mat], b = xs->offs[mat + 1];
    double sig = orc_sigma_t(xs->E + a, xs->S + a, b - a, (double)E);
    sig_out[s] = sig;
    score_out[s] = segment_score(wt, tau, sig, lens[s]);
    tau += sig * lens[s];
  }
  return ns;
}

/* ------------------------------------------------------------------ */
/* whole batch                                                          */
/* ------------------------------------------------------------------ */

static void atomic_add_double(double *addr, double val) {
  uint64_t *ptr = (uint64_t *)addr;
  uint64_t old = __atomic_load_n(ptr, __ATOMIC_RELAXED);
  for (;;) {
    double cur;
    memcpy(&cur, &old, sizeof cur);
    double nv = cur + val;
    uint64_t nbits;
    memcpy(&nbits, &nv, sizeof nbits);
    if (__atomic_compare_exchange_n(ptr, &old, nbits, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED))
      return;
  }
}

typedef struct {
  const orc_mesh *m;
  const orc_xs *xs;
  const double *edges;
  int32_t n_groups;
  const float *r[8]; /* x y z u v w E wt */
  int64_t begin, end;
  double *tally;     /* shared tally (atomic adds) or private tally */
  int use_atomic;
  int64_t segments;  /* positive-length segments scored */
  int64_t rejected;  /* rays that score nothing because of bad fields */
  int64_t overflow;  /* rays whose walk exceeded the step bound */
} orc_job;

static void *cast_worker(void *arg) {
  orc_job *j = (orc_job *)arg;
  const orc_mesh *m = j->m;
  const int64_t cap = (int64_t)m->nx + m->ny + m->nz + 3;
  const int64_t ncells = (int64_t)m->nx * m->ny * m->nz;
  int64_t *cells = (int64_t *)malloc(sizeof(int64_t) * cap);
  double *tin = (double *)malloc(sizeof(double) * cap);
  double *lens = (double *)malloc(sizeof(double) * cap);
  double *sig = (double *)malloc(sizeof(double) * (j->xs->n_materials + 1));
  for (int64_t r = j->begin; r < j->end; ++r) {
    const float E = j->r[6][r], wt = j->r[7][r];
    double p[3], d[3];
    if (!prepare_ray(j->r[0][r], j->r[1][r], j->r[2][r], j->r[3][r], j->r[4][r], j->r[5][r], E,
                     wt, p, d)) {
      j->rejected++;
      continue;
    }
    int32_t g = orc_group(j->edges, j->n_groups, (double)E);
    if (g < 0) continue;
    int64_t ns = orc_trace_dda(m, p, d, cells, tin, lens, cap);
    if (ns < 0) { j->overflow++; continue; }
    for (int32_t k = 0; k < j->xs->n_materials; ++k) {
      const int64_t a = j->xs->offs[k], b = j->xs->offs[k + 1];
      sig[k] = orc_sigma_t(j->xs->E + a, j->xs->S + a, b - a, (double)E);
    }
    double *t = j->tally + (int64_t)g * ncells;
    double tau = 0.0;
    for (int64_t s = 0; s < ns; ++s) {
      double sg = sig[m->material[cells[s]]];
      double sc = segment_score(wt, tau, sg, lens[s]);
      tau += sg * lens[s];
      if (lens[s] > 0.0) j->segments++;
      if (j->use_atomic) atomic_add_double(t + cells[s], sc);
      else t[cells[s]] += sc;
    }
  }
  free(cells); free(tin); free(lens); free(sig);
  return NULL;
}

int32_t orc_hardware_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int32_t)n : 1;
}

/* Adds the Eq. 4 scores of n rays to tally[n_groups * ncells] (which the
 * caller zeroes or seeds).  nthreads <= 0 uses every online core.  Small
 * tallies are accumulated in per-thread copies and summed; large ones with
 * atomic compare-and-swap adds.  Returns 0, or -1 on allocation failure.
 * stats (may be NULL) receives {segments, rejected rays, overflowed rays,
 * threads used}. */
int32_t orc_cast(const orc_mesh *m, const orc_xs *xs, const double *edges, int32_t n_groups,
                 const float *x, const float *y, const float *z, const float *u, const float *v,
                 const float *w, const float *E, const float *wt, int64_t n, double *tally,
                 int32_t nthreads, int64_t *stats) {
  if (nthreads <= 0) nthreads = orc_hardware_threads();
  if (n < (int64_t)nthreads * 64) nthreads = (int32_t)(n / 64 > 0 ? n / 64 : 1);
  const int64_t G = (edges == NULL || n_groups <= 0) ? 1 : n_groups;
  const int64_t tsize = G * (int64_t)m->nx * m->ny * m->nz;
  const int privatize = nthreads > 1 && (double)tsize * nthreads * 8.0 <= 512.0 * 1024 * 1024;
  orc_job *jobs = (orc_job *)calloc((size_t)nthreads, sizeof(orc_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -1; }
  for (int32_t i = 0; i < nthreads; ++i) {
    orc_job *j = &jobs[i];
    j->m = m; j->xs = xs; j->edges = edges; j->n_groups = n_groups;
    j->r[0] = x; j->r[1] = y; j->r[2] = z; j->r[3] = u;
    j->r[4] = v; j->r[5] = w; j->r[6] = E; j->r[7] = wt;
    j->begin = n * i / nthreads;
    j->end = n * (i + 1) / nthreads;
    if (privatize) {
      j->tally = (double *)calloc((size_t)tsize, sizeof(double));
      if (!j->tally) { for (int32_t q = 0; q < i; ++q) free(jobs[q].tally); free(jobs); free(th); return -1; }
      j->use_atomic = 0;
    } else {
      j->tally = tally;
      j->use_atomic = nthreads > 1;
    }
  }
  for (int32_t i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, cast_worker, &jobs[i]);
  cast_worker(&jobs[0]);
  for (int32_t i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
  int64_t seg = 0, rej = 0, ovf = 0;
  for (int32_t i = 0; i < nthreads; ++i) {
    seg += jobs[i].segments;
    rej += jobs[i].rejected;
    ovf += jobs[i].overflow;
    if (privatize) {
      for (int64_t c = 0; c < tsize; ++c) tally[c] += jobs[i].tally[c];
      free(jobs[i].tally);
    }
  }
  if (stats) { stats[0] = seg; stats[1] = rej; stats[2] = ovf; stats[3] = nthreads; }
  free(jobs);
  free(th);
  return 0;
}

/* ------------------------------------------------------------------ */
/* next-event (point-detector) estimator                                */
/* ------------------------------------------------------------------ */

/* Flux at n_det detector points from every ray event, assuming isotropic
 * emission: wt * exp(-tau) / (4 pi R^2), with R the distance from the event
 * to the detector and tau the optical depth along that straight line
 * (vacuum outside the mesh).  The event direction is not used.  An event
 * exactly at a detector (R = 0) contributes nothing.  Adds to
 * out[det][group] (n_det x n_groups, group layout as the tally). */
int32_t orc_point_detector(const orc_mesh *m, const orc_xs *xs, const double *edges,
                           int32_t n_groups, const float *x, const float *y, const float *z,
                           const float *E, const float *wt, int64_t n, const double *det,
                           int32_t n_det, double *out) {
  const int64_t cap = (int64_t)m->nx + m->ny + m->nz + 3;
  const int32_t G = (edges == NULL || n_groups <= 0) ? 1 : n_groups;
  int64_t *cells = (int64_t *)malloc(sizeof(int64_t) * cap);
  double *tin = (double *)malloc(sizeof(double) * cap);
  double *lens = (double *)malloc(sizeof(double) * cap);
  double *sig = (double *)malloc(sizeof(double) * (xs->n_materials + 1));
  if (!cells || !tin || !lens || !sig) { free(cells); free(tin); free(lens); free(sig); return -1; }
  for (int64_t r = 0; r < n; ++r) {
    if (!isfinite(x[r]) || !isfinite(y[r]) || !isfinite(z[r]) || !isfinite(E[r]) ||
        !isfinite(wt[r]) || !(E[r] > 0.0f))
      continue;
    const int32_t g = orc_group(edges, n_groups, (double)E[r]);
    if (g < 0) continue;
    for (int32_t k = 0; k < xs->n_materials; ++k) {
      const int64_t a = xs->offs[k], b = xs->offs[k + 1];
      sig[k] = orc_sigma_t(xs->E + a, xs->S + a, b - a, (double)E[r]);
    }
    const double p[3] = {x[r], y[r], z[r]};
    for (int32_t k = 0; k < n_det; ++k) {
      double d[3] = {det[3 * k] - p[0], det[3 * k + 1] - p[1], det[3 * k + 2] - p[2]};
      const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (!(R > 0.0)) continue;
      d[0] /= R; d[1] /= R; d[2] /= R;
      const int64_t ns = orc_trace_dda(m, p, d, cells, tin, lens, cap);
      double tau = 0.0;
      for (int64_t s = 0; s < ns; ++s) {
        if (tin[s] >= R) break;
        const double l = (tin[s] + lens[s] > R) ? R - tin[s] : lens[s];
        tau += sig[m->material[cells[s]]] * l;
      }
      out[(int64_t)k * G + g] += (double)wt[r] * exp(-tau) / (4.0 * M_PI * R * R);
    }
  }
  free(cells); free(tin); free(lens); free(sig);
  return 0;
}
