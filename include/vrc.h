/*
 * vrc.h - C ABI of libvrc, a GB300 (sm_103a) implementation of the
 * volumetric-ray-casting (VRC) fluence estimator of Sweezy,
 * "A Monte Carlo Volumetric-Ray-Casting Estimator for Global Fluence
 * Tallies on GPUs" (arXiv:1706.07476).
 *
 * A batch of ray events (position, direction, energy, weight) handed over by
 * a CPU random walk is traced through a 3-D Cartesian mesh of material
 * cells.  Every crossed cell i receives the expected track length of Eq. 4,
 *
 *     s_i = wt * exp(-tau_in) * (1 - exp(-Sigma_t,i(E) l_i)) / Sigma_t,i(E)
 *
 * (wt * exp(-tau_in) * l_i in void), where tau_in is the optical depth from
 * the ray start to the entry of cell i (the integral of Eq. 2) and wt is the
 * per-ray weight W/N of Eq. 4.  Scores accumulate in a device-resident
 * tally that is copied back on request (Sec. 3: the tally stays on the GPU
 * until the end of the run).
 *
 * Conventions shared by every call:
 *  - Return value: VRC_OK (0) or a negative VRC_ERR_* code.  No C++
 *    exception crosses this boundary.  vrc_last_error() returns a
 *    thread-local message describing the last failure on the calling thread.
 *  - Ownership: a vrc_ctx owns all device memory it allocates and every copy
 *    of caller data it makes.  The caller keeps ownership of its own arrays.
 *  - Streams: a `cuda_stream` argument is a cudaStream_t passed as void*;
 *    NULL selects the context's own stream.
 *  - Units: lengths in cm, energies in eV, cross sections in 1/cm.
 *  - Floating point: rays are float32; mesh geometry, energy grids and the
 *    tally are float64.
 */
#ifndef VRC_H
#define VRC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define VRC_OK 0
#define VRC_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, bad table) */
#define VRC_ERR_STATE (-2)     /* call out of order, e.g. cast before a used material has data */
#define VRC_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define VRC_ERR_OOM (-4)       /* device or pinned-host allocation failed */
#define VRC_ERR_TRAVERSAL (-5) /* a ray needed more grid steps than nx+ny+nz+3 */
#define VRC_ERR_NONFINITE (-6) /* a ray had a non-finite field, energy <= 0 or a zero direction */

/* ---- precision forms -------------------------------------------------- */
/* PLAIN: the paper's arithmetic (Sec. 3): single-precision cross sections
 * and distances, Eq. 4 evaluated in double precision, float64 tally.
 * Distances are computed with double-float (two float32) arithmetic; each
 * segment's e^-x and e^-x - 1 are within 0.6 and 2 ulp of the exact
 * values.  A ray stops scoring once its optical depth passes
 * 760 + ln(max(wt, 1)), where wt e^-tau is below the float64 range (any
 * score dropped there is below 1e-322).
 * FP32: Eq. 4's exponentials and the optical depth in float32 (optical depth
 * kept as a compensated float32 pair); the tally sums stay float64. */
#define VRC_FORM_PLAIN 0
#define VRC_FORM_FP32 1

/* ---- flags for vrc_read_tally ---------------------------------------- */
#define VRC_PER_VOLUME 1 /* divide each cell's tally by the cell volume dx*dy*dz */

typedef struct vrc_ctx vrc_ctx;

/* Tuning and behaviour options.  vrc_default_options() fills the defaults;
 * any field left at its "auto" value is chosen by the library. */
typedef struct {
  int32_t form;           /* VRC_FORM_PLAIN (default) or VRC_FORM_FP32 */
  int32_t sort;           /* counting sort of the rays by (energy group, number of cells
                             crossed) before the cast: 0 off, 1 on, -1 auto (on for batches
                             of 65,536 rays or more; default) */
  int32_t sort_len_buckets; /* crossed-cell buckets per group in the sort key, 1..256;
                               -1 auto (256, fewer when groups x buckets would pass 16,384) */
  int32_t block;          /* threads per block of the cast kernel; 0 auto */
  int32_t blocks_per_sm;  /* resident blocks per SM for the cast grid; 0 auto */
  int32_t device;         /* CUDA device ordinal for this context; -1 = current device */
  int32_t stop_at_zero;   /* 1: a ray's walk ends once its transmitted fraction exp(-tau) is
                             exactly 0 in the form's precision (every later score would be +0,
                             so the tally is bit for bit the same up to summation order); the
                             segment counter then counts only the walked segments.  0 (default):
                             every ray is walked to the mesh exit, as the paper casts it */
  int32_t rays_per_warp;  /* how the cast kernel hands rays to its warps: -1 interleaved (warp w
                             of the persistent grid takes rays w*32 + lane, then the next 32 rays
                             one grid further); R > 0, a multiple of 32 up to 65,536: each warp
                             takes R consecutive (sorted) rays at a time from a device counter,
                             so warps that finish early take more work; 0 auto (default:
                             32 in the plain form and for FP32 casts of 2^23 rays or more,
                             interleaved for smaller FP32 casts) */
} vrc_options;

/* A uniform 3-D Cartesian mesh (Sec. 3: 3-D Cartesian mesh geometry).
 * Cell (ix, iy, iz) spans [x0 + ix*dx, x0 + (ix+1)*dx) x ... ; outside the
 * box is vacuum (Sec. 5.1).  `material` is a HOST array of nx*ny*nz ids in
 * [0, n_materials), x fastest ([iz][iy][ix]); it is copied.  n_materials is
 * at most 64.  Energy groups: n_groups >= 1; group_edges is a HOST array of
 * n_groups+1 strictly ascending energies (eV), group g = [e_g, e_g+1), last
 * group closed, rays outside every group score nothing; group_edges == NULL
 * requires n_groups == 1 and takes every energy.  Tally layout:
 * [group][iz][iy][ix] float64. */
typedef struct {
  int32_t nx, ny, nz;
  double x0, y0, z0;
  double dx, dy, dz;
  const uint8_t *material;
  int32_t n_materials;
  int32_t n_groups;
  const double *group_edges;
} vrc_mesh_desc;

/* A batch of n rays as eight float32 arrays (structure of arrays).  Each is
 * a device pointer when on_device != 0, else a host pointer.  (u, v, w) need
 * not be normalised (only the direction is used); wt already carries the
 * 1/N of Eq. 4. */
typedef struct {
  const float *x, *y, *z;
  const float *u, *v, *w;
  const float *E;
  const float *wt;
  int64_t n;
  int32_t on_device;
} vrc_rays;

/* Counters accumulated on the device since the last reset. */
typedef struct {
  int64_t segments;   /* ray-cell segments with positive length that were scored */
  int64_t rays;       /* rays processed (including those that scored nothing) */
  int64_t rejected;   /* rays rejected as VRC_ERR_NONFINITE */
  int64_t overflow;   /* rays stopped by the step bound (VRC_ERR_TRAVERSAL) */
  int64_t live;       /* segments whose score was added (non-zero): once a ray's transmitted
                         fraction exp(-tau) is exactly 0 in the form's precision, its later
                         segments are walked and counted in `segments` but add nothing */
} vrc_stats;

/* Fills *opt with the defaults.  Never fails. */
void vrc_default_options(vrc_options *opt);

/* Creates a context for one mesh (Sec. 3: MonteRay holds the mesh geometry
 * and the cross sections).  Copies the mesh to the device and allocates a
 * zeroed tally of n_groups*nx*ny*nz float64.  opt may be NULL (defaults).
 * On failure *out is NULL and nothing is leaked.
 * Errors: VRC_ERR_ARG (null pointer, non-positive or non-finite size or
 * spacing, material id >= n_materials, n_materials outside 1..64, bad group
 * edges), VRC_ERR_OOM, VRC_ERR_CUDA. */
int vrc_create_mesh(const vrc_mesh_desc *d, const vrc_options *opt, vrc_ctx **out);

/* A rectilinear (non-uniform Cartesian) mesh, the structured meshes of the
 * Sec. 6 outlook: cell (ix, iy, iz) spans [x_edges[ix], x_edges[ix+1]) x
 * [y_edges[iy], y_edges[iy+1]) x [z_edges[iz], z_edges[iz+1]).  Each edge
 * array is a HOST array of n+1 finite, strictly ascending float64 plane
 * positions (cm), copied; every other field means what it does in
 * vrc_mesh_desc.  The walk takes each crossing from the plane positions
 * (kept on the device as double-float pairs, about 48 bits). */
typedef struct {
  int32_t nx, ny, nz;
  const double *x_edges, *y_edges, *z_edges;
  const uint8_t *material;
  int32_t n_materials;
  int32_t n_groups;
  const double *group_edges;
} vrc_rect_mesh_desc;

/* vrc_create_mesh for a rectilinear mesh.  Every call on the context works
 * as on a uniform mesh (VRC_PER_VOLUME divides by each cell's own volume),
 * except vrc_detector_flux and the batched form, which return VRC_ERR_ARG.
 * Errors: as vrc_create_mesh, and VRC_ERR_ARG for NULL, non-finite or
 * non-ascending edges. */
int vrc_create_rect_mesh(const vrc_rect_mesh_desc *d, const vrc_options *opt, vrc_ctx **out);

/* Loads the total macroscopic cross-section table of one material (Sec. 3:
 * continuous-energy total cross sections, linearly interpolated between
 * table points; clamped to the end values outside the table).  E_eV and
 * sigma_t are HOST arrays of n float64 values, copied.  n == 0 makes the
 * material void (sigma_t = 0).  Loading a material again replaces its table.
 * Errors: VRC_ERR_ARG (material out of range, n < 0, null arrays with n > 0,
 * energies not strictly ascending, non-finite or non-positive energies,
 * negative or non-finite sigma). */
int vrc_load_xs(vrc_ctx *c, int32_t material, const double *E_eV, const double *sigma_t,
                int64_t n);

/* Casts a batch of rays and adds their Eq. 4 scores to the tally (Sec. 3:
 * per ray, cross-section lookup, ray cast, VRC score).  Asynchronous on the
 * stream: device arrays must stay valid until the stream passes this point.
 * With sorting on, the rays are first copied, in sorted order, into
 * context-owned scratch (36 B per ray plus a small table); the tally is the
 * same up to float64 summation order.
 * Host arrays (on_device == 0) are copied to the device before the call
 * returns.  A host batch of more than 2^22 rays is uploaded in chunks (2^21
 * rays, then up to 2^24) on a context-owned copy stream, each chunk sorted
 * and cast on cuda_stream while the next one uploads (two 512 MiB staging
 * slots); pinned host arrays make these copies asynchronous.  Rays with a
 * non-finite field, E <= 0 or a zero direction score
 * nothing and are reported by the next vrc_sync / vrc_read_tally as
 * VRC_ERR_NONFINITE.  n == 0 is a no-op.
 * Errors: VRC_ERR_ARG, VRC_ERR_STATE (a material used by the mesh has no
 * table), VRC_ERR_OOM (a scratch buffer could not be allocated; the call
 * takes every buffer before it launches a kernel, so it has added nothing),
 * VRC_ERR_CUDA. */
int vrc_cast_rays(vrc_ctx *c, const vrc_rays *r, void *cuda_stream);

/* Sorts a device batch of rays the way vrc_cast_rays does before its cast
 * (by energy group, then by the number of cells crossed) without allocating
 * any memory.  The paper has no counterpart: it is for callers that may not
 * call cudaMalloc once their run has started, e.g. a transport code that
 * gives all free device memory to its own pool at start-up, or one whose
 * batch loop must not pay the device-wide synchronisation of cudaMalloc /
 * cudaFree while the CPU random walk keeps running.  Cast the result with
 * sorting off (options.sort = 0) to get vrc_cast_rays' sorted cast.
 *  - in: device rays (on_device != 0), at most 262,144 per call; larger
 *    batches are rejected with VRC_ERR_ARG (split them).
 *  - out: caller-owned device array of 8*n floats receiving the sorted rays
 *    as x, y, z, u, v, w, E, wt blocks of n each.
 *  - the key uses the context's mesh box, groups and sort_len_buckets.
 *  - scratch: one fixed device array of about 5 MiB inside libvrc, shared by
 *    every call; each call writes all of it that it reads, so nothing needs
 *    clearing.  Calls that overlap on the GPU (other streams, other threads,
 *    other contexts on the same device) race on it: serialise them.
 *  - set-up: the first call on each device looks up the scratch's device
 *    address (cudaGetSymbolAddress) and makes the sort kernels resident.
 *    Under CUDA's lazy module loading (the default) that is when the driver
 *    places the array and the kernels' code on the device, which can
 *    allocate device memory; the device then holds them until the process
 *    exits.  Make that first call before the caller's pool takes the
 *    device's free memory, and before any stream capture; every later call
 *    on that device allocates nothing.
 *  - asynchronous on cuda_stream (NULL = the context's stream).
 * Errors: VRC_ERR_ARG (NULL pointers, host rays, too many rays or keys),
 * VRC_ERR_CUDA. */
int vrc_sort_rays_static(vrc_ctx *c, const vrc_rays *in, float *out, void *cuda_stream);

/* Waits for the stream and reports the device status accumulated since the
 * last reset: VRC_ERR_NONFINITE or VRC_ERR_TRAVERSAL if any ray hit that
 * case (the tally still holds every other ray's scores), else VRC_OK.
 * stats may be NULL. */
int vrc_sync(vrc_ctx *c, void *cuda_stream, vrc_stats *stats);

/* Copies the tally (n must equal n_groups*nx*ny*nz) to the HOST array
 * out_host, layout [group][iz][iy][ix], optionally divided by the cell
 * volume (VRC_PER_VOLUME).  Synchronous: waits for all work queued on the
 * context's stream and on cuda_stream.  Returns the device status like
 * vrc_sync (the copy is made in every case unless the error is ARG/CUDA). */
int vrc_read_tally(vrc_ctx *c, double *out_host, int64_t n, int32_t flags, void *cuda_stream);

/* Device pointer of the float64 tally (n_groups*nx*ny*nz entries) for
 * callers that reduce or post-process it on the device; valid until
 * vrc_destroy.  NULL if c is NULL. */
double *vrc_tally_device_ptr(vrc_ctx *c);

/* The context's own stream (a cudaStream_t as void*): the stream that a NULL
 * cuda_stream selects in every call on this context, and in vrc_batch_*
 * calls on a batch whose first context this is.  A caller that produces
 * device rays on another stream orders this one after it (an event and
 * cudaStreamWaitEvent) before the call that reads them.  Owned by the
 * context and valid until vrc_destroy; NULL if c is NULL. */
void *vrc_context_stream(vrc_ctx *c);

/* Zeroes the tally, the counters and the device status (stream-ordered on
 * cuda_stream). */
int vrc_reset_tally(vrc_ctx *c, void *cuda_stream);

/* Replaces the context's options (form, sort, launch shape). */
int vrc_set_options(vrc_ctx *c, const vrc_options *opt);

/* Frees every resource of the context; NULL is a no-op. */
void vrc_destroy(vrc_ctx *c);

/* Thread-local description of the last error ("" if none). */
const char *vrc_last_error(void);

/* ---- next-event (point-detector) estimator -----------------------------
 * Sec. 6 names moving the next-event estimator to the GPU as future work.
 * For every ray event (position, energy, weight; its direction is not used)
 * and every detector point, adds wt * exp(-tau) / (4 pi R^2) to
 * out[detector][group]: isotropic emission, R the distance from the event to
 * the detector, tau the optical depth along that straight line through the
 * mesh (vacuum outside).  An event exactly at a detector adds nothing.
 * Rays: device or host arrays as in vrc_cast_rays.  det_xyz: HOST array of
 * n_det (1..64) points (float64, rounded to float32 on the device).  out:
 * HOST array of n_det * n_groups float64, overwritten.  Synchronous.  Does
 * not touch the tally.  Errors: VRC_ERR_ARG, VRC_ERR_STATE, VRC_ERR_OOM,
 * VRC_ERR_CUDA; VRC_ERR_TRAVERSAL if a walk hit the step bound. */
int vrc_detector_flux(vrc_ctx *c, const vrc_rays *r, const double *det_xyz, int32_t n_det,
                      double *out, void *cuda_stream);

/* ---- tally statistics: batches or histories ----------------------------
 * The figure of merit (Eq. 5) and the fractional difference (Eq. 8) need the
 * standard deviation of each cell's tally.  Two ways to get it, both ending
 * in running sums S1 = sum_b x_b and S2 = sum_b x_b^2 over B samples, after
 * which the tally total is S1 and its standard deviation
 * sqrt(B/(B-1) (S2 - S1^2/B)):
 *  - VRC_MOMENTS_BATCH: a sample is the tally of one batch of histories.  The
 *    caller casts one batch (for example one filled ray buffer) with
 *    vrc_cast_rays, then vrc_moments_fold moves the tally into S1/S2.
 *  - VRC_MOMENTS_HISTORY: a sample is one history's score x_h.  Each ray
 *    carries the id of its history; vrc_cast_histories sums the scores of a
 *    history's rays per cell and adds x_h to S1 and x_h^2 to S2.  With the
 *    1/N of Eq. 4 folded into wt, this sigma is the usual Monte Carlo
 *    standard deviation of the tally mean over N histories. */
#define VRC_MOMENTS_OFF 0
#define VRC_MOMENTS_BATCH 1
#define VRC_MOMENTS_HISTORY 2

/* Allocates (mode BATCH or HISTORY) or frees (OFF) the moment array, one
 * float64 (S1, S2) pair per tally entry (twice the tally's size), and zeroes
 * it and the sample count.  Waits for the context's stream.  VRC_ERR_ARG for
 * another mode. */
int vrc_moments_enable(vrc_ctx *c, int32_t mode);

/* S1 += tally, S2 += tally^2, tally = 0, sample count + 1 (stream-ordered).
 * VRC_ERR_STATE unless the mode is VRC_MOMENTS_BATCH. */
int vrc_moments_fold(vrc_ctx *c, void *cuda_stream);

/* Per-history cast (mode VRC_MOMENTS_HISTORY, else VRC_ERR_STATE).
 * history[i] (uint32) is the history of ray i, on the same side as the rays
 * (device if r->on_device, else host); the rays of one history may sit
 * anywhere in the call, but a history must not continue in a later call.
 * n_histories is the number of histories the call completes, counting those
 * without rays (their score is zero); it is added to the sample count.
 * Scores go to S1/S2 only: the tally is untouched.  The tabulated cross
 * sections are used (not the surrogate); the rays are sorted as in
 * vrc_cast_rays (options.sort), their history ids with them.
 * Needs (group count x cells) < 2^32 - 1.  How: each ray writes its scores
 * as (history, bin, score) records into its own stretch of a pair buffer,
 * sized by an upper bound of its segments; the records are sorted into
 * buckets of consecutive bins, and per bucket the scores of each (history,
 * bin) are summed in shared memory and folded into S1/S2.  Device scratch,
 * kept for later calls: two pair buffers, 12 B per ray, the bucket table,
 * and the sorted copy of the rays and of their ids (36 B per ray).  With
 * device inputs the pair buffers are sized for every ray's largest bound,
 * 16 B x n x (nx + ny + nz + 10) each (13 GB for 2^20 rays in a 256^3
 * mesh), when both fit in a quarter of the free device memory: the call
 * then never waits on the device (it synchronises the stream only when it
 * grows them).  Otherwise, and always with host inputs, the call waits for
 * the sum of its rays' bounds (one small device-to-host read) and sizes the
 * buffers to 16 B per bound segment (about 3 GB each for 2^20 rays crossing
 * 256^3 cells); VRC_ERR_OOM when they do not fit or when that bound passes
 * 2^32 - 1 segments (split the call).  The cast and the fold into S1/S2 are
 * queued on cuda_stream (NULL = the context's stream).  Host arrays may be
 * reused on return; device arrays must stay valid until the stream passes
 * the call. */
int vrc_cast_histories(vrc_ctx *c, const vrc_rays *r, const uint32_t *history, int64_t n_histories,
                       void *cuda_stream);

/* Synchronous: total = S1 and sigma = sqrt(B/(B-1) (S2 - S1^2/B)) per
 * (group, cell) into HOST arrays of n = n_groups*nx*ny*nz float64 (sigma may
 * be NULL; sigma is 0 with fewer than 2 samples); *samples receives B (the
 * batch or history count).  Reports a per-history overflow (a ray with
 * more segments than its bound, or a bucket whose keys overflow the
 * shared-memory table) as VRC_ERR_OOM. */
int vrc_moments_read(vrc_ctx *c, double *total, double *sigma, int64_t n, int64_t *samples,
                     void *cuda_stream);

/* ---- streaming ray buffers ---------------------------------------------
 * Sec. 3: the CPU random walk stores rays in a buffer; when it is full the
 * buffer goes to the GPU and is cleared, and the CPU keeps simulating
 * histories while the GPU casts it (Secs. 2-3: the casting cost hides behind
 * the random walk).  A vrc_stream keeps n_buffers pinned host buffers of
 * 32-byte ray records: the producer fills one while earlier ones are copied
 * (on a copy stream) and cast (on the context's stream), the two ordered by
 * events so that a buffer is reused only after its copy, and its device
 * copy only after its cast, have finished. */
typedef struct {
  float x, y, z, u, v, w, E, wt;
} vrc_ray_record;

typedef struct vrc_stream vrc_stream;

/* Allocates n_buffers (>= 2) pinned host buffers and device buffers of
 * capacity rays each for context c.  Errors: VRC_ERR_ARG, VRC_ERR_OOM,
 * VRC_ERR_CUDA. */
int vrc_stream_create(vrc_ctx *c, int64_t capacity, int32_t n_buffers, vrc_stream **out);

/* Hands out the next pinned host buffer to fill (capacity records); waits
 * until that buffer's previous upload has finished.  Calling acquire twice
 * without a submit returns the same buffer. */
int vrc_stream_acquire(vrc_stream *s, vrc_ray_record **buffer, int64_t *capacity);

/* Queues the first n records of the acquired buffer: asynchronous H2D copy,
 * then the cast into the context's tally.  Returns at once. */
int vrc_stream_submit(vrc_stream *s, int64_t n);

/* Waits until every submitted buffer has been cast. */
int vrc_stream_finish(vrc_stream *s);

/* Waits for the stream's work and frees its buffers; NULL is a no-op. */
void vrc_stream_destroy(vrc_stream *s);

/* ---- learned cross-section surrogate ------------------------------------
 * Energy is constant along a ray (Eq. 4 has one E_j per ray), so Σt of every
 * material is needed once per ray.  The surrogate replaces the table lookup
 * (Sec. 3: hashed search, lin-lin interpolation) by a small network
 * evaluated on the tensor cores:
 *   x = (log10 E - log10 e_lo)/(log10 e_hi - log10 e_lo);
 *   features sin(pi f_k x), cos(pi f_k x), f_k = 2^(5k/31), k = 0..31;
 *   h1 = silu(W1 x + b1) (64->128); h2 = silu(W2 h1 + b2) (128->128);
 *   y = W3 h2 + b3 + log(a + b E^(-1/2)) (128->16), y_m = log Σt of material m.
 * The last term is a fixed per-material prior, the 1/v shape of a total
 * cross section (a_m > 0, b_m >= 0), fitted to the table before training;
 * the network learns the rest.
 * Parameters: VRC_MLP_PARAMS float32 values, W1 [128][64], b1 [128],
 * W2 [128][128], b2 [128], W3 [16][128], b3 [16], C [16][2] (a_m, b_m).
 * W1 and W2 are rounded to bfloat16 and run on the tensor cores with float32
 * accumulation; their inputs (the features and h1) enter as bfloat16 pairs
 * hi + lo (about 16 significant bits); the output layer runs in float32
 * (W3 and h2 float32).  The exact table stays the fallback: after training,
 * every hash bin whose validated relative error exceeds the bound is flagged
 * and rays in flagged bins use the table. */
#define VRC_MLP_PARAMS 26928
#define VRC_XS_TABLE 0
#define VRC_XS_SURROGATE 1

/* Forward pass: log Σt of 16 outputs for n energies.  All pointers are
 * DEVICE arrays: params [VRC_MLP_PARAMS], E [n], log_sigma [n][16].  e_lo and
 * e_hi set the input normalisation.  Asynchronous on cuda_stream. */
int vrc_mlp_forward(const float *params, const float *E, int64_t n, double e_lo, double e_hi,
                    float *log_sigma, void *cuda_stream);

/* Loss and gradient: loss = (1/count) Σ over unmasked (row, output) pairs of
 * (y - target)^2 and its gradient with respect to params (the prior's
 * coefficients included).  DEVICE arrays: target [n][16], mask [n][16]
 * (uint8, non-zero = used; NULL = all used), grad [VRC_MLP_PARAMS] and
 * loss [1] (both overwritten).  count = number of used pairs (> 0). */
int vrc_mlp_loss_grad(const float *params, const float *E, const float *target,
                      const uint8_t *mask, int64_t n, int64_t count, double e_lo, double e_hi,
                      float *grad, float *loss, void *cuda_stream);

typedef struct {
  int32_t steps;   /* Adam steps (default 12000); 0 keeps the trained parameters and only
                      re-validates them at tol (VRC_ERR_STATE if none exist) */
  int32_t batch;   /* rows per step (default 4096) */
  float lr;        /* peak learning rate, cosine decay (default 5e-3) */
  float tol;       /* accepted relative error of Σt per hash bin (default 1e-3) */
  uint64_t seed;   /* initial weights and row sampling (default 4) */
  float smooth;    /* training uses only the table intervals where log Σt of every
                      material stays within this of a straight line in log E over 7
                      union-grid points (default 5e-6); resonance structure stays with
                      the table */
} vrc_surrogate_options;

typedef struct {
  float final_loss;            /* mean squared error of the normalised targets, last step */
  int32_t bins, bins_accepted; /* hash bins, and bins where the surrogate is used */
  float coverage;              /* bins_accepted / bins */
  float max_rel_err_accepted;  /* largest validated relative Σt error in accepted bins */
  float median_rel_err;        /* median validated relative Σt error over all points */
  int64_t train_points, validation_points;
  float smooth_fraction;       /* fraction of union-grid intervals trained on */
} vrc_surrogate_report;

void vrc_default_surrogate_options(vrc_surrogate_options *opt);

/* Trains the context's surrogate on its own tables with libvrc's kernels
 * (forward, backward, Adam): fits each material's prior, trains the network
 * on the smooth intervals (see vrc_surrogate_options.smooth), then validates
 * it at 8 energies per union-grid interval that are not training points, and
 * flags every hash bin (with its two neighbours) where any material's
 * relative Σt error exceeds tol or that holds no validation point.  At most
 * 16 materials; void materials are not modelled (Σt = 0 exactly); if a
 * non-void table has a zero Σt, no bin is accepted.  Synchronous.  Does not
 * change the lookup mode.  report may be NULL.
 * Errors: VRC_ERR_ARG, VRC_ERR_STATE (no tables), VRC_ERR_OOM, VRC_ERR_CUDA. */
int vrc_train_surrogate(vrc_ctx *c, const vrc_surrogate_options *opt, vrc_surrogate_report *report);

/* Selects VRC_XS_TABLE (default) or VRC_XS_SURROGATE for later casts
 * (VRC_ERR_STATE if no surrogate has been trained).  With the surrogate, a
 * cast always sorts its rays, those whose energy lies in an accepted bin
 * first; the network runs on exactly those rays (one tensor-core forward
 * pass, Σt of all materials into context scratch of 64 B per ray) and every
 * other ray uses the table.  With no bin accepted the network does no work. */
int vrc_set_xs_mode(vrc_ctx *c, int32_t mode);

/* Copies the trained parameters (VRC_MLP_PARAMS float32) to a HOST array. */
int vrc_get_surrogate_params(vrc_ctx *c, float *params_host);

/* ---- batched form ------------------------------------------------------
 * Many independent tally problems (each a context with its own mesh, cross
 * sections and tally, and its own device ray batch) cast by ONE persistent
 * kernel that takes chunks of rays ("work items") from a device counter, the
 * whole launch sequence captured once in a CUDA graph.  This generalises the
 * paper's one-problem GPU step (Sec. 3) to serving many problems at once; the
 * per-ray arithmetic is that of vrc_cast_rays (Eq. 4). */
typedef struct vrc_batch vrc_batch;

typedef struct {
  int32_t block;            /* threads per block: 0 auto (256), else 32..256 step 32 */
  int32_t blocks_per_sm;    /* resident blocks per SM: 0 auto (occupancy) */
  int32_t chunk;            /* rays per work item: 0 auto (2048), else 64..65536 */
  int32_t sort_len_buckets; /* 0: no sort; 1..256: sort each problem's rays by (group,
                               crossed cells) into this many buckets first; -1 auto (16) */
  int32_t use_graph;        /* 1 (default): capture the sequence in a CUDA graph once */
  int32_t rays_per_warp;    /* how a block hands a work item's rays to its warps: 0 (default)
                               interleaved (warp w takes rays w*32 + lane, then one block
                               further); R > 0, a multiple of 32 up to 8,192: each warp takes R
                               consecutive rays at a time from the item's counter in shared
                               memory, so warps that finish early take more of the item */
} vrc_batch_options;

void vrc_default_batch_options(vrc_batch_options *opt);

/* Builds a batch plan over n_problems contexts.  rays[p] is problem p's
 * DEVICE ray batch (on_device != 0); the arrays must stay valid and
 * unchanged in size for the plan's lifetime (their contents may change
 * between launches).  All contexts must live on one device and use the same
 * precision form.  Uploads any pending cross sections, allocates the plan's
 * device state (work list, problem table, optional sort scratch of 36 B per
 * ray) and, with use_graph, captures the sequence.
 * Errors: VRC_ERR_ARG (NULL, host rays, mixed devices or forms, more than
 * 2^31 work items or 2^32 rays), VRC_ERR_STATE (missing cross sections),
 * VRC_ERR_OOM, VRC_ERR_CUDA. */
int vrc_batch_create(vrc_ctx *const *ctxs, const vrc_rays *rays, int32_t n_problems,
                     const vrc_batch_options *opt, vrc_batch **out);

/* Casts every problem's rays into its own context's tally: one graph launch
 * (or the plain launch sequence) on cuda_stream (NULL = the first context's
 * stream).  Asynchronous; use vrc_sync / vrc_read_tally on each context. */
int vrc_batch_launch(vrc_batch *b, void *cuda_stream);

/* Frees the plan (waits for its launches); NULL is a no-op. */
void vrc_batch_destroy(vrc_batch *b);

/* One-shot: create a plan with default options, launch it, wait, destroy. */
int vrc_cast_batched(vrc_ctx *const *ctxs, const vrc_rays *rays, int32_t n_problems,
                     void *cuda_stream);

/* Kernel timing.  When enabled, every cast records CUDA events on the
 * launching stream around its kernels; vrc_get_timing waits for the stream
 * and returns the summed device time (ms) of the cast kernels and of the ray
 * sort kernels, and the number of cast-kernel launches, since timing was
 * enabled or last read with reset != 0. */
int vrc_enable_timing(vrc_ctx *c, int32_t on);
int vrc_get_timing(vrc_ctx *c, void *cuda_stream, double *cast_ms, double *sort_ms,
                   int64_t *cast_launches, int32_t reset);

/* Number of kernels libvrc has launched in this process (all contexts). */
int64_t vrc_launch_count(void);

/* Failure injection for tests (no counterpart in the paper): with n >= 0,
 * the next n device or pinned-host allocations libvrc makes (in any call,
 * any thread) succeed and the one after fails as if the device were out of
 * memory, without asking the driver; the hook then disarms itself.  n < 0
 * disarms it.  The failing call returns VRC_ERR_OOM: a create call then
 * returns NULL and leaks nothing, and a cast adds nothing to the tally (a
 * cast takes all its buffers before it launches anything, also a large host
 * batch cast in chunks).  Touches no GPU; always returns VRC_OK. */
int vrc_debug_fail_alloc(int64_t n);

/* Number of CUDA devices visible (0 when none or on failure). */
int vrc_device_count(void);

/* Library version as major*10000 + minor*100 + patch (0.4.0: the
 * allocation-failure hook vrc_debug_fail_alloc; 0.3.0: vrc_options
 * gained rays_per_warp and vrc_stats gained live; 0.2.0: vrc_options gained
 * stop_at_zero; rectilinear meshes, per-history moments, the next-event
 * estimator and streaming buffers were added). */
#define VRC_VERSION 400
int vrc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VRC_H */
