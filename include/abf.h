/*
 * abf.h -- adaptive box-spline filtering on one GPU (GB300, sm_103a).
 *
 * The operation (Chaudhury, Munoz-Barrutia, Unser, "Fast adaptive elliptical
 * filtering using box splines"):
 *
 *   Sec. 6:  s[m] = < f, beta^4_{a(m)}( . - m) >  for every pixel m, where
 *            beta^4_a is the four-direction box spline of Sec. 4 Eq. (def)
 *            (N = 4, theta_k = (k-1) pi/4) and f is the image with phi = delta
 *            (Sec. 7 (1)).
 *   Sec. 7:  computed as a global pre-integration (four running-sum recursions,
 *            Eq. (RS)) followed, per pixel, by the affine finite-difference mesh
 *            of Eq. (final_eqn) / Table "Mesh Vertices" with ZP interpolation.
 *
 * Order n (1..3) applies every directional box n times (the n-fold running sum
 * Delta_b^{-n} of Sec. 2 and the FD filter d^n_a of Eq. (FD)); the mesh then has
 * (n+1)^4 vertices and the interpolation kernel is ZP^{*n}.  n = 1 is Sec. 7.
 *
 * Units.  Scales enter as lattice steps c_k: the k-th box is the segment c_k v_k
 * with v = (1,0), (1,1), (0,1), (-1,1); c1 = a1, c3 = a3, c2 = a2/sqrt2,
 * c4 = a4/sqrt2 in the paper's scales (its a'_j).  Steps are rounded to the
 * 2^-Q grid: C_k = rint(c_k 2^Q), ties to even.
 *
 * Boundary.  The image is zero outside [0, W) x [0, H) (zero padding).
 *
 * Conventions for every entry point below:
 *   - pointers named d_* are DEVICE pointers allocated and owned by the caller;
 *     the library never frees them.  Images are row-major, row pitch in BYTES.
 *   - calls are asynchronous on the given cudaStream_t (0 = legacy default);
 *     the returned status covers argument checks and launch errors.  Errors
 *     found on the device (invalid scales, range overflow, a bounded wait
 *     that ran out) set a status word that abf_last_device_status() reads.
 *   - no exceptions cross the ABI; no call aborts the process.
 *   - there is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns ABF_ERR_CUDA.
 */
#ifndef ABF_H
#define ABF_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ABF_OK = 0,
  ABF_ERR_INVALID = 1,      /* bad argument or descriptor                         */
  ABF_ERR_OOM = 2,          /* device or host allocation failed                   */
  ABF_ERR_CUDA = 3,         /* CUDA runtime error (no device, launch failure)     */
  ABF_ERR_UNSUPPORTED = 4,  /* valid request the library does not serve          */
  ABF_ERR_RANGE = 5,        /* exact form: numerator would exceed 64*limbs bits   */
  ABF_ERR_TIMEOUT = 6,      /* a bounded device or host wait ran out              */
  ABF_ERR_BUSY = 7          /* serving: admission refused (over the HBM budget)   */
} abf_status;

typedef enum { ABF_U8 = 0, ABF_U16 = 1, ABF_F32 = 2, ABF_F64 = 3 } abf_dtype;

typedef enum {
  /* Exact: running sums in wrap-around integers modulo 2^(64 L) (L limbs),
   * integer ZP^{*n} weights, integer numerator S; one binary64 division at the
   * end.  Bit-exact numerator.  Input must be integer after scaling by 2^F.  */
  ABF_FORM_EXACT = 0,
  /* Plain: running sums restarted on a window around each output tile (the
   * window holds every read of the tile's mesh), then the mesh, all in pairs
   * of binary64 numbers (hi + lo, error-free TwoSum / TwoProd: unit roundoff
   * about 2^-104).  Every pixel checks an a-priori bound on its error; where
   * it exceeds 1e-12 times the plan's value bound the pixel is NaN and sets
   * ABF_DEV_PRECISION.  Single binary64 cannot meet 1e-12: the mesh cancels
   * the running sums by up to 1e13 (order 2, steps 1..150).               */
  ABF_FORM_PLAIN_F64 = 1,
  /* As PLAIN_F64 in pairs of binary32 numbers (unit roundoff about 2^-46),
   * tolerance 1e-5 times the value bound.  Order 1 only: at order 2 and 3
   * the bound exceeds 1e-5 already for the smallest window that holds one
   * pixel's reads at unit steps, so the plan returns ABF_ERR_UNSUPPORTED.  */
  ABF_FORM_TILE_F32 = 2
} abf_form;

typedef enum {
  ABF_SCALES_C4 = 0,      /* float32 x4 per pixel: lattice steps c1..c4              */
  ABF_SCALES_A4 = 1,      /* float32 x4 per pixel: paper scales a1..a4 (Sec. 7)      */
  ABF_SCALES_ELLIPSE = 2  /* float32 x4 per pixel: sigma, elongation, cos t, sin t   */
} abf_scale_kind;

/* Descriptor of one filtering problem (image size, order, types, form). */
typedef struct {
  int32_t width, height;      /* image size in pixels (>= 1)                          */
  int32_t order_n;            /* n in {1, 2, 3}                                       */
  int32_t in_dtype;           /* abf_dtype of f                                       */
  int32_t out_dtype;          /* ABF_F32 or ABF_F64                                   */
  int32_t form;               /* abf_form                                             */
  int32_t scale_kind;         /* abf_scale_kind                                       */
  int32_t q_bits;             /* Q: steps on the 2^-Q grid (1..9 for n = 1, else 1..8) */
  int32_t in_frac_bits;       /* F: f 2^F is an integer (exact form); 0 for u8/u16    */
  int32_t flags;              /* 0 or ABF_FLAG_DEBUG_BOUNDS                           */
  double max_scale;           /* upper bound on every step c_k (lattice units)        */
  double min_scale;           /* lower bound on c1 and c3 (>= 2^-Q); 0 means 1.0      */
  double value_bound;         /* upper bound on |f|; 0 means the dtype's range (u8,   *
                               * u16 only: required for float inputs)                 */
  double max_scale_product;   /* upper bound on c1 c2 c3 c4; 0 means max_scale^4      */
  /* Directional order N of Sec. 4 Eq. (def): 0 or 4 (theta = 0, pi/4, pi/2,
   * 3pi/4; Sec. 7), or 2 (theta = 0, pi/2: tensor box splines, the other
   * member of the family whose running-sum filters of Eq. (RS_filter) lie on
   * the lattice).  With N = 2 only c1 and c3 shape the kernel; c2 and c4 are
   * read and must be valid; order n >= 2 unless a model is used (n = 1 alone
   * is a discontinuous box); scale kinds c4 and a4 only.                    */
  int32_t directions;
  /* Image model of Sec. 6, f(x) = sum_k c[k] phi(x - k): 0 for phi = delta
   * (Sec. 7 (1)); E >= 1 for the tensor B-spline phi = beta^{E-1} (x)
   * beta^{E-1} (E unit boxes per axis, E <= 6).  For E >= 3 the coefficients
   * c = f * (b^{E-1})^-1 are irrational and are rounded to the 2^-F grid
   * (c_q = rint(c 2^F)) by a separable prefilter in abf_integrate; the rest
   * is exact on c_q.  Models and N = 2 need q_bits <= 7 and the exact form. */
  int32_t model_boxes;
} abf_desc;

typedef struct abf_plan_s* abf_plan;

/* Create a plan for the problem of Sec. 6 (s[m] = <f, beta_{a(m)}(. - m)> for
 * a given per-pixel scale map) with the four-direction box spline of Sec. 7,
 * phi = delta (Sec. 7 (1)) and order n (each directional box n-fold): host
 * work + one upload of the ZP^{*n} weight table, which is shared by all plans
 * with the same n and grid.  The plan fixes the lattice
 * box of the integrated image: [-left, W + right) x [0, H + above) in image
 * coordinates (rows below the image are all zero and are not stored).
 * Errors: ABF_ERR_INVALID (descriptor), ABF_ERR_RANGE (exact form: the
 * numerator bound needs more than 4 limbs), ABF_ERR_CUDA / ABF_ERR_OOM.      */
abf_status abf_plan_create(const abf_desc* desc, abf_plan* out);
/* Free the plan's own memory (the plan and its device status word); the
 * weight tables, shared by plans, stay with the library until the process
 * exits, and caller buffers are never touched.  ABF_ERR_INVALID for NULL.    */
abf_status abf_plan_destroy(abf_plan plan);

/* Sizes the caller allocates (the lattice box of the non-adaptive step of
 * Sec. 7 (1)): the integrated image (exact form; 0 otherwise)
 * and the scratch workspace; the margins (left, right, below, above) of the
 * integrated lattice box; the number of 64-bit limbs L (exact form) and the
 * row pitch of the integrated image in elements (each element L * 8 bytes).
 * Any output pointer may be NULL.                                            */
abf_status abf_plan_query(abf_plan plan, size_t* integrated_bytes, size_t* workspace_bytes,
                          int32_t* halo_lrbt, int32_t* limbs, int64_t* g_pitch_elems);

/* Host-only: the interpolation table of a generalised plan (directions N,
 * order n, model_boxes E; Eq. (mask): the box spline with the lattice
 * directions v1..v4 taken (n + E, n, n + E, n) times, or (n + E, 0, n + E, 0)
 * for N = 2) on the 2^-P grid, P = q_bits + 1, without touching a device.
 * Layout: (2^P)^2 rows, row index ry 2^P + rx for the offset r = (rx, ry) 2^-P
 * of a tap from its floor point; each row holds D M(r - d) for the *R
 * neighbours d, listed in stencil_xy as (dx, dy) pairs (caller array of 512
 * int32); *wbytes-byte little-endian words.  With out = NULL only the sizes,
 * the stencil and D are returned.                                           */
abf_status abf_general_table_host(int32_t directions, int32_t n, int32_t model_boxes, int32_t q_bits, void* out,
                                  size_t out_bytes, size_t* needed_bytes, int32_t* wbytes, int32_t* R,
                                  int32_t* stencil_xy, uint32_t* D_words4);

/* Non-adaptive step (Sec. 7 (1), Eq. (RS)) of the exact form: the four
 * running-sum recursions, each n times, in the paper's order (0, pi/4, pi/2,
 * 3pi/4), unit weights (the paper's sqrt2 factors are folded into the
 * normaliser), modulo 2^(64 L).
 *   d_f   : H rows of W elements of desc.in_dtype, row pitch f_pitch bytes.
 *   d_g   : integrated image, abf_plan_query() bytes, layout
 *           g[(k2) * pitch + (k1 + left)][limb] (uint64 limbs, little-endian),
 *           k2 in [0, H + above).  Equal to the exact running sums wherever the
 *           3pi/4 recursion's backward ray leaves the box through its bottom
 *           row; elsewhere it differs from them by a polynomial of degree < n
 *           along each 3pi/4 line, which the mesh annihilates.
 *   d_ws  : workspace of abf_plan_query() bytes (scan carries and flags),
 *           any contents: the call clears what must start at zero.  It may be
 *           reused by any plan afterwards, but two calls that overlap on the
 *           GPU must not share it.                                           */
abf_status abf_integrate(abf_plan plan, const void* d_f, size_t f_pitch, void* d_g,
                         void* d_ws, cudaStream_t stream);

/* abf_integrate without a caller workspace, for callers that cannot allocate
 * device memory: for example a serving loop whose memory is reserved once, up
 * front, by a caching allocator it may not step around, or code that must not
 * risk the implicit device synchronisation of cudaMalloc / cudaFree.  The paper
 * has no counterpart: this is an interface for such callers only.
 *
 * The scan carries and flags use a fixed scratch array inside the library
 * (32 MiB, a static device array that every GPU loading the library holds until
 * the process exits).  The call allocates nothing; the caller still supplies
 * d_f and d_g exactly as for abf_integrate.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any
 *     stream capture.  The address is kept for the life of the process: after
 *     cudaDeviceReset on that device the cached address is stale, so do not
 *     call this entry point again in a process that reset the device.
 *   - The current device must be the plan's device (else ABF_ERR_INVALID).
 *   - Plans whose workspace (abf_plan_query) exceeds 32 MiB are rejected with
 *     ABF_ERR_UNSUPPORTED (e.g. order 2, two limbs, steps up to 150: images up
 *     to about 3300 x 3300).
 *   - Every call shares the one array and clears the parts that must start at
 *     zero; calls that overlap on the GPU (other streams, other threads) race
 *     on it and give wrong results: serialise them.                          */
abf_status abf_integrate_noalloc(abf_plan plan, const void* d_f, size_t f_pitch, void* d_g,
                                 cudaStream_t stream);

/* Adaptive step (Eq. (final_eqn)) for every pixel.
 *   exact form:      d_src = the integrated image from abf_integrate().
 *   PLAIN_F64 / TILE_F32: d_src = the image f itself (pitch f_pitch bytes);
 *                    the running sums are restarted per output tile; d_ws is
 *                    the plan's workspace (abf_plan_query); pixels whose
 *                    error bound exceeds the form's tolerance get NaN and set
 *                    ABF_DEV_PRECISION.
 *   d_scales : H rows of W float4 (desc.scale_kind), row pitch in bytes.
 *   d_s      : H rows of W desc.out_dtype, row pitch in bytes.
 * Pixels whose scales are invalid (non-finite, C_k = rint(c_k 2^Q) < 1 or
 * > rint(max_scale 2^Q), c1 or c3 < min_scale) or whose numerator bound
 * exceeds the limbs get NaN and set the device status.                       */
abf_status abf_filter(abf_plan plan, const void* d_src, size_t src_pitch, const void* d_scales,
                      size_t scale_pitch, void* d_s, size_t s_pitch, void* d_ws,
                      cudaStream_t stream);

/* Exact form only: the numerator of Eq. (final_eqn) before the normaliser,
 * as integers S[m] = D sum_j w_j g_I(y_j)
 * (L uint64 limbs per pixel, two's complement modulo 2^(64 L)), row pitch in
 * bytes.  s[m] = S[m] 2^(4 Q n) / (D (C1 C2 C3 C4)^n 2^F).                    */
abf_status abf_filter_numerator(abf_plan plan, const void* d_g, const void* d_scales,
                                size_t scale_pitch, void* d_num, size_t num_pitch, void* d_ws,
                                cudaStream_t stream);

/* One image of a batched non-adaptive step: its (exact-form) plan, image,
 * integrated image and workspace, exactly as the arguments of abf_integrate. */
typedef struct {
  abf_plan plan;
  const void* d_f;
  size_t f_pitch;
  void* d_g;
  void* d_ws;
} abf_integrate_job;

/* Non-adaptive step (Sec. 7 (1), Eq. (RS)) of many images of uneven size,
 * order, limbs and input type: the images of one (limbs, order, input type)
 * group share one row-pass launch (a CTA per row of any of them) and one
 * launch per line direction (v2, v3, v4) whose CTAs take bands of any image
 * from one ticket counter, image by image and band by band within an image.
 * Every image's integrated image is bit-identical to abf_integrate on it
 * alone.  One extra launch clears all images' look-back flags first.
 *   jobs  : njobs entries (host memory, read during the call); each image's
 *           d_ws is its own plan workspace, as for abf_integrate, and must not
 *           be shared with a call that overlaps on the GPU.
 *   d_ws  : at least 256 bytes of device memory (the ticket counters).
 * Batches of more than abf_integrate_batch_max_jobs() images are split into
 * several calls' worth of launches.  Device errors go to each image's plan
 * status word.                                                              */
abf_status abf_integrate_batch(const abf_integrate_job* jobs, int32_t njobs, void* d_ws, size_t ws_bytes,
                               cudaStream_t stream);
int32_t abf_integrate_batch_max_jobs(void);

/* One image of a batch: its (exact-form) plan, its integrated image from
 * abf_integrate, its scale field and its output (as for abf_filter).        */
typedef struct {
  abf_plan plan;
  const void* d_g;
  const void* d_scales;
  size_t scale_pitch;
  void* d_s;
  size_t s_pitch;
} abf_job;

/* Adaptive step (Eq. (final_eqn)) for many images of uneven size, order and
 * limb count in one persistent launch per (order n, limbs) present: the
 * images' row runs (32 pixels of one row) are numbered (largest images first,
 * within an image band by band and strip by strip) and every warp takes the
 * next run from a device counter on its own, so the work stays balanced
 * across SMs with no barrier between runs.  Each image's result is
 * bit-identical to abf_filter on that image alone.
 *   jobs  : njobs entries (host memory, read during the call), every plan of
 *           the exact form; up to abf_batch_max_jobs() per call (larger
 *           batches are split into several launches).
 *   d_ws  : device workspace of at least 256 bytes (the work counters); two
 *           calls that overlap on the GPU must not share it.
 * Device errors go to each job's plan status word.                           */
abf_status abf_filter_batch(const abf_job* jobs, int32_t njobs, void* d_ws, size_t ws_bytes,
                            cudaStream_t stream);
int32_t abf_batch_max_jobs(void);

/* Autotuner (no counterpart in the paper: a launch-shape choice).  The exact
 * mesh runs a CTA over R consecutive rows of 32-pixel runs (R warps; their
 * taps share g patches in L1).  These calls time R = 4, 8, 16 on the caller's
 * own data (one untimed and one timed run each, CUDA events on `stream`,
 * which they synchronise) and keep the fastest: abf_plan_autotune in the plan
 * (used by later abf_filter / abf_filter_numerator calls), abf_batch_autotune
 * in a process-wide cache keyed by the batch's composition (the sorted
 * (n, limbs, width, height) of its images; used by later abf_filter_batch
 * calls on batches of that composition).  Outputs are written as by
 * abf_filter / abf_filter_batch.  *warps_out = the choice; ms3 (optional):
 * the three times in ms.  Choices are also kept process-wide by key (GPU
 * name, order, limbs, size, Q and scale kind for a plan; GPU name and the
 * composition for a batch) and, when the environment variable
 * ABF_TUNE_CACHE names a file, in that file (a flat JSON object
 * {"key": rows}, read at the first lookup, rewritten after every tuning):
 * abf_plan_create starts an exact plan from a kept choice for its key.
 * abf_plan_rows reports a plan's current rows per CTA.                      */
abf_status abf_plan_autotune(abf_plan plan, const void* d_g, const void* d_scales, size_t scale_pitch, void* d_s,
                             size_t s_pitch, cudaStream_t stream, int32_t* warps_out, float* ms3);
abf_status abf_batch_autotune(const abf_job* jobs, int32_t njobs, void* d_ws, size_t ws_bytes, cudaStream_t stream,
                              int32_t* warps_out, float* ms3);
abf_status abf_plan_rows(abf_plan plan, int32_t* rows);

/* ------------------------------------------------------------------ serving
 * No counterpart in the paper: a serving interface around its two steps
 * (Sec. 6, (1) non-adaptive and (2) adaptive).  A request loop for filter jobs (image + per-pixel scale field, host memory)
 * on one GPU.  A worker thread admits queued jobs in arrival order as long as
 * a slot (a CUDA stream) is free and the job's device footprint (image,
 * scales, output, integrated image, workspace) fits the HBM budget; later
 * jobs that fit may pass a head job that does not.  Admitted jobs run
 * concurrently on their streams (copy in, abf_integrate, abf_filter, copy out),
 * so jobs that arrive while others run overlap with them on the device.
 * Integrated images can stay resident under an image id: a later job with the
 * same id and the same descriptor skips the copy of the image and the
 * non-adaptive step (filtering the same image with a new scale field).
 * Resident images are evicted least-recently-used when memory is needed.
 * Results are the same as abf_integrate + abf_filter on the job alone.      */
typedef struct abf_server_s* abf_server;

/* Server flag: the jobs admitted together (in one round of the worker) run
 * their adaptive step in one batched launch (as abf_filter_batch) after each
 * has finished its own copies and non-adaptive step on its own stream.      */
#define ABF_SERVER_GROUP_MESH 1

typedef struct {
  size_t hbm_budget;        /* bytes of device memory the server may hold (> 0)    */
  int32_t max_inflight;     /* jobs running at once (slots, 1..64)                  */
  int32_t flags;            /* 0 or ABF_SERVER_GROUP_MESH                           */
} abf_server_cfg;

typedef struct {
  abf_desc desc;            /* exact form                                           */
  const void* h_f;          /* host image (pinned memory lets copies overlap)       */
  size_t f_pitch;
  const void* h_scales;     /* host scale field, H x W float4                       */
  size_t scale_pitch;
  void* h_s;                /* host output, H x W desc.out_dtype                    */
  size_t s_pitch;
  uint64_t image_id;        /* 0: do not keep; else keep the integrated image       */
} abf_request;

typedef struct {
  double t_submit_us, t_admit_us, t_done_us;  /* host steady clock, microseconds  */
  int32_t resident_hit;     /* 1 if the integrated image was reused                 */
  int32_t status;           /* abf_status of the job (valid once done)              */
  int32_t device_status;    /* OR of ABF_DEV_* bits raised by this job's own launches */
  int32_t reserved;
  /* Device clock (CUDA events on the job's stream), microseconds since the
   * server was created: when the job's first copy could start and when its
   * last copy ended.  Two jobs whose intervals intersect were on the device
   * at the same time.  0 if the job never ran.                              */
  double t_gpu_start_us, t_gpu_end_us;
} abf_job_stats;

/* Start a server on the current device.  Errors: ABF_ERR_INVALID, ABF_ERR_CUDA. */
abf_status abf_server_create(const abf_server_cfg* cfg, abf_server* out);
/* Queue a job; the host buffers must stay valid until the job is done.
 * ABF_ERR_BUSY if the job alone exceeds the budget.  A request with h_f =
 * NULL must name an image that is resident now (else ABF_ERR_INVALID); that
 * image is then held (never evicted) until the job is done.                 */
abf_status abf_submit(abf_server srv, const abf_request* req, uint64_t* ticket);
/* done = 1 once the job finished (stats filled); the record is kept until waited. */
abf_status abf_poll(abf_server srv, uint64_t ticket, int32_t* done, abf_job_stats* stats);
/* Wait up to timeout_us (< 0: no limit) for a job; ABF_ERR_TIMEOUT if it is not
 * done by then (the job stays queued or running).  Releases the record when done. */
abf_status abf_wait(abf_server srv, uint64_t ticket, int64_t timeout_us, abf_job_stats* stats);
/* Stop (1) or resume (0) admitting queued jobs; running jobs continue.     */
abf_status abf_server_pause(abf_server srv, int32_t paused);
/* Bytes held now / at most so far, jobs running, jobs queued, resident images. */
abf_status abf_server_stats(abf_server srv, size_t* used, size_t* peak, int32_t* inflight,
                            int32_t* queued, int32_t* resident);
/* Finish every queued and running job, then free everything.               */
abf_status abf_server_destroy(abf_server srv);

/* The per-pixel integer steps C_k = rint(c_k 2^Q) (int32 x4 per pixel) that
 * abf_filter uses, for inspection and reuse: the scale reading of Sec. 7
 * (c2 = a2 / sqrt2, c4 = a4 / sqrt2, the a'_j of Table "Mesh Vertices") or the
 * ellipse moment rule (a reading; its isotropic case is Theorem (convergence)
 * of Sec. 4).  d_C: H rows of W int4, row pitch C_pitch bytes.  Invalid pixels
 * get zeros and set the device status.                                       */
abf_status abf_prepare_scales(abf_plan plan, const void* d_scales, size_t scale_pitch,
                              void* d_C, size_t C_pitch, cudaStream_t stream);

/* Measure a scale field before planning (no counterpart in the paper: the
 * bounds that size a plan's limbs): the largest step max_k c_k and the
 * largest product c1 c2 c3 c4 over the image, after rounding to the 2^-Q grid
 * (desc supplies width, height, order_n, scale_kind, q_bits and max_scale, the
 * clamp of the ellipse rule).  Synchronises `stream`.  Returns
 * ABF_ERR_INVALID if some pixel's scales are invalid.  Allocates 24 bytes of
 * device memory for the duration of the call.                               */
abf_status abf_measure_scales(const abf_desc* desc, const void* d_scales, size_t scale_pitch,
                              double* max_step, double* max_product, cudaStream_t stream);

/* The common denominator D of the integer ZP^{*n} weights of this plan (the
 * interpolation weights of Eq. (final_eqn) are D times the kernel's values on
 * the 2^-P grid), as four 32-bit words (little-endian, D < 2^128).          */
abf_status abf_plan_denominator(abf_plan plan, uint32_t* d_words4);

/* Read and clear the plan's device status word (synchronises the device; no
 * counterpart in the paper).  code = 0 or an OR of ABF_DEV_* bits.           */
#define ABF_DEV_BAD_SCALE   1   /* a scale was non-finite, non-positive or out of bounds */
#define ABF_DEV_RANGE       2   /* a pixel's numerator bound exceeded 64 L - 1 bits       */
#define ABF_DEV_TIMEOUT     4   /* a bounded wait (scan look-back) ran out                 */
#define ABF_DEV_BAD_INPUT   8   /* f 2^F not an integer within value_bound (exact form)   */
#define ABF_DEV_PRECISION  16   /* floating-point forms: a pixel's error bound exceeded the
                                   form's tolerance (the pixel is NaN)                     */
#define ABF_DEV_BOUNDS     32   /* ABF_FLAG_DEBUG_BOUNDS: a tap's reads left the lattice box */
abf_status abf_last_device_status(abf_plan plan, int32_t* code);

/* Bounds checking of the adaptive step (no counterpart in the paper: a check
 * of the lattice box the plan sizes from Sec. 7's reach of the taps).  A plan
 * created with abf_desc.flags = ABF_FLAG_DEBUG_BOUNDS (exact form) runs
 * abf_filter / abf_filter_numerator with checked kernels: before any read,
 * every tap's lattice point plus the order's stencil box (generalised plans:
 * each lane's neighbour at the extreme taps of the pixel) must lie inside the
 * lattice box (columns 0 .. Gw - 1, rows up to Gh - 1; rows below 0 are zero
 * by definition and never read).  Reads that would leave it are not made (the
 * tap, or that lane's share of the pixel, adds nothing), the status word gets
 * ABF_DEV_BOUNDS and the first such pixel (first in device order) is
 * recorded.  abf_debug_bounds_violation returns that pixel as y W + x, or -1
 * if none, and clears the record (synchronises the device).  Returns
 * ABF_ERR_INVALID for a plan created without the flag.  Batched launches
 * (abf_filter_batch, grouped serving) and plans without the flag run the
 * unchecked kernels.  ABF_ERR_UNSUPPORTED for the floating-point forms.     */
#define ABF_FLAG_DEBUG_BOUNDS 1
abf_status abf_debug_bounds_violation(abf_plan plan, int64_t* pixel);

/* Host-side fault injection (no counterpart in the paper; failure detection
 * is tested without faulting a GPU).  Arms `count` faults of one kind,
 * process-wide; count = 0 disarms it.
 *   ABF_FAULT_ALLOC       the next `count` device allocations of plan
 *                         creation (abf_plan_create: ABF_ERR_OOM, nothing
 *                         leaked) and of server jobs (the job ends with
 *                         ABF_ERR_OOM) fail;
 *   ABF_FAULT_QUEUE_STALL while armed the server admits no queued job (as if
 *                         their publication were withheld): abf_wait runs
 *                         into its timeout; disarming lets the jobs run;
 *   ABF_FAULT_BAD_DESC    the next `count` abf_plan_create calls (also those a
 *                         server makes for its jobs) see an invalid
 *                         descriptor: ABF_ERR_INVALID.
 * The environment variable ABF_FAULT (read once, at the library's first
 * plan or server call) arms the same: a comma-separated list of
 * kind[:count] with kind alloc, queue_stall or bad_desc (count 1 if omitted).
 * Returns ABF_ERR_INVALID for an unknown kind or a negative count.          */
#define ABF_FAULT_ALLOC        1
#define ABF_FAULT_QUEUE_STALL  2
#define ABF_FAULT_BAD_DESC     3
abf_status abf_debug_inject_fault(int32_t kind, int32_t count);

const char* abf_status_str(abf_status s);

/* Host-only: generate the ZP^{*n} weight table (the interpolation kernel of
 * Eq. (final_eqn): the ZP element of Sec. 7, n-fold self-convolved) for order
 * n and grid 2^-Q (the table abf_plan_create uploads) into a caller buffer, without touching a
 * device.  Layout: (2^P)^2 rows, row index ry 2^P + rx (P = Q for even n,
 * Q + 1 for odd n; fractional offset r = (rx, ry) 2^-P, minus 1/2 for odd n).
 * Row entries: D ZP^{*n}(r - d) for the lattice neighbours d that can carry a
 * non-zero weight (9, 32, 69 of the (3n)^2 candidates for n = 1, 2, 3), in
 * [dy][dx] order, dx, dy from d_min = -3n/2 + 1 (n even) or -(3n - 1)/2
 * (n odd); the dropped candidates are those whose box of r - d misses the
 * open support |x|, |y| < 3n/2, |x +- y| < 2n.  Little-endian words of
 * *wbytes bytes (4, 8 or 16).
 * With out = NULL only *needed_bytes, *wbytes and D are returned.            */
abf_status abf_weight_table_host(int32_t n, int32_t q_bits, void* out, size_t out_bytes,
                                 size_t* needed_bytes, int32_t* wbytes, uint32_t* D_words4);

/* --------------------------------------------------- scale-map estimation
 * The paper leaves the scale map a: Z^2 -> R^4_+ to other work (Sec. 8).  This
 * builds one from the image (a reading, not the paper's): the
 * structure tensor J = G_rho * (g g^T) of the central-difference gradient g
 * (zero outside the image; sampled Gaussian of std rho, |k| <= ceil(3 rho),
 * normalised, applied separably in binary32), its eigenvalues l1 >= l2 and
 * coherence ((l1 - l2) / (l1 + l2 + 1e-12))^2 (binary64), and per pixel the
 * ellipse (sigma0, 1 + (e_max - 1) coherence, cos t, sin t) with (cos t, sin t)
 * the unit eigenvector of l2, sin t >= 0 ((1, 0) where l1 == l2): the input of
 * ABF_SCALES_ELLIPSE, so the filter smooths along edges.
 *   d_f   : height rows of width in_dtype elements, row pitch in bytes.
 *   d_ws  : device workspace of abf_ellipse_ws_bytes(width, height) bytes.
 *   d_out : height rows of width float4, row pitch in bytes (16-aligned).
 *   rho in (0, 10], sigma0 > 0, e_max >= 1.                                 */
size_t abf_ellipse_ws_bytes(int32_t width, int32_t height);
abf_status abf_estimate_ellipses(const void* d_f, size_t f_pitch, abf_dtype in_dtype, int32_t width, int32_t height,
                                 double rho, double sigma0, double e_max, void* d_ws, size_t ws_bytes, void* d_out,
                                 size_t out_pitch, cudaStream_t stream);

/* ------------------------------------------------- 1-D adaptive filter (Sec. 3)
 *
 * The scale-adaptive B-spline filter of Sec. 3 (Proposition "prop") on a batch
 * of 1-D signals (rows): s[m] = < f, beta_{a(m)}^{n2}( . - m) > with the model
 * f(x) = sum_k c[k] beta^{n1}(x - k), beta_a^n(x) = beta^n(x / a) / a.  For
 * n1 in {0, 1} the interpolation prefilter is the identity (c = f) and the
 * result is exact: g = n2+1 causal running sums of c in wrap-around integers,
 * then per sample the FD mask Delta_a^{n2+1} with degree N = n1+n2+1 B-spline
 * interpolation at y_j = m + tau - a j, tau = (a-1)(n2+1)/2 (Eq. (link)):
 *   S[m] = sum_j (-1)^j binom(n2+1, j) sum_k g[k] D beta^N(y_j - k),
 *   s[m] = S[m] 2^(Q (n2+1)) / (D A^(n2+1) 2^F),  D = N! 2^(N (Q+1)),
 * with A = rint(a 2^Q).  The signal is zero outside [0, length).
 * For n1 in 2..5 the model coefficients c = f * (b^{n1})^-1 (b^{n1}[k] =
 * beta^{n1}(k), the B-spline interpolation filter; the inverse is two-sided
 * and irrational) are rounded to the 2^-F grid, c_q = rint(c 2^F), and the
 * two steps run exactly on c_q, which starts `left` samples before the signal
 * (its decaying tail).  Since the kernel of s in terms of c is non-negative
 * with unit lattice sum, |s - s(c)| <= 2^-(F+1) plus the prefilter's own
 * error (binary64 poles and weights in 64-bit fixed point: about
 * 2^-46 |f|max 2^F + 2^-18 grid steps), which can only move c_q by one step
 * where c 2^F lies that close to a rounding tie.
 * n1 >= 6 returns ABF_ERR_UNSUPPORTED.                                       */
typedef struct {
  int32_t length;         /* samples per signal, >= 1                           */
  int32_t count;          /* signals (rows), >= 1                               */
  int32_t n1;             /* model degree: 0..5                                 */
  int32_t n2;             /* analysis degree: 0..3                              */
  abf_dtype in_dtype;     /* f elements                                         */
  abf_dtype out_dtype;    /* s elements: ABF_F32 or ABF_F64                     */
  int32_t q_bits;         /* Q: scales rounded to the 2^-Q grid, 1..10          */
  int32_t in_frac_bits;   /* F: float f must lie on the 2^-F grid (0 for ints)  */
  double max_scale;       /* bound on every a (>= 2^-Q)                         */
  double value_bound;     /* bound on |f|; 0 = dtype range (integer inputs)     */
} abf1d_desc;

typedef struct abf1d_plan_s* abf1d_plan;

/* Plan: validates the descriptor, picks the limb count L from the numerator
 * bound D max_scale^(n2+1) |c|max 2^F (|s| <= |c|max: the kernel is
 * non-negative with unit lattice sum; |c|max = |f|max for n1 <= 1, else
 * ||(b^{n1})^-1||_1 |f|max), uploads the D beta^N table.  For n1 >= 2 the
 * plan also owns a staging buffer for c_q (count x g_pitch_elems int32, or
 * int64 when ||(b^{n1})^-1||_1 |f|max 2^F does not fit 31 bits).
 * ABF_ERR_RANGE if L would exceed 4, or (n1 >= 2) if |f|max 2^F leaves fewer
 * than 24 guard bits in the prefilter's 64-bit fixed point (about 2^35).    */
abf_status abf1d_plan_create(const abf1d_desc* desc, abf1d_plan* out);
abf_status abf1d_plan_destroy(abf1d_plan plan);

/* Sizes of the Proposition's step 1 output.
 * integrated_bytes: size of the integrated signals g (count rows of
 * g_pitch_elems elements of L uint64 limbs; element i holds g at signal
 * position i - left); left: samples before the signal start that g holds (0
 * for n1 <= 1); right: samples past the signal end that g holds (the adaptive
 * step reads up to tau + (N+1)/2 beyond it).  Any pointer may be NULL.      */
abf_status abf1d_plan_query(abf1d_plan plan, size_t* integrated_bytes, int32_t* left, int32_t* right,
                            int32_t* limbs, int64_t* g_pitch_elems);

/* Non-adaptive step (Proposition "prop", step 1, Sec. 3):
 * g = u_1^{(n2+1)} * (c 2^F) per row, exact modulo
 * 2^(64 L) (c = f for n1 <= 1; the prefiltered c_q for n1 >= 2).  d_f: count
 * rows of length in_dtype elements (row pitch in bytes); d_g: plan-sized,
 * 16-byte aligned.  Off-grid or out-of-bound float inputs read as 0 and set
 * ABF_DEV_BAD_INPUT.  Launches: the prefilter (n1 >= 2), then the row pass.  */
abf_status abf1d_integrate(abf1d_plan plan, const void* d_f, size_t f_pitch, void* d_g, cudaStream_t stream);

/* Adaptive step (Proposition "prop", step 2, Sec. 3: the FIR localisation
 * mask Delta_a^{n2+1} beta^{n1+n2+1}(k + tau)): d_a holds one float32 scale a
 * per sample (count rows, row
 * pitch in bytes); d_s receives s (out_dtype).  Samples whose scale is
 * invalid (non-finite, A < 1 or A > rint(max_scale 2^Q)) or whose numerator
 * bound exceeds the limbs get NaN and set the device status.                 */
abf_status abf1d_filter(abf1d_plan plan, const void* d_g, const float* d_a, size_t a_pitch, void* d_s,
                        size_t s_pitch, cudaStream_t stream);

/* Step 2 before the normaliser a^-(n2+1): the integer numerators S[m] (L
 * little-endian uint64 limbs per sample, two's
 * complement modulo 2^(64 L)), for bit-exact checks.                         */
abf_status abf1d_filter_numerator(abf1d_plan plan, const void* d_g, const float* d_a, size_t a_pitch,
                                  void* d_num, size_t num_pitch, cudaStream_t stream);

/* Device status bits (ABF_DEV_*; no counterpart in the paper) of the plan's
 * launches since the last read;
 * synchronises the device, then clears the word.                             */
abf_status abf1d_last_device_status(abf1d_plan plan, int32_t* code);

/* Host-only: the B-spline weight table abf1d_plan_create uploads (the
 * interpolation by beta^N of the Proposition's step 2, Sec. 3), without
 * touching a device.  2^(Q+1) rows (r = R 2^-(Q+1) in [0, 1)) of *K entries
 * D beta^N(r - d), d = *dmin .. *dmin + *K - 1, N = n1 + n2 + 1,
 * D = N! 2^(N (Q+1)).  With out = NULL only the sizes and D are returned.   */
abf_status abf1d_weight_table_host(int32_t n1, int32_t n2, int32_t q_bits, uint64_t* out, size_t out_elems,
                                   size_t* needed_elems, int32_t* K, int32_t* dmin, uint64_t* D);

/* Host-only: the constants of the interpolation prefilter c = f * (b^{n1})^-1
 * (Sec. 3) that abf1d_plan_create derives for n1 in 2..5: the inverse of the
 * B-spline interpolation filter as h[k] = sum_p A_p z_p^|k| over *npoles
 * (1 or 2) poles z_p in (-1, 0), binary64; z and A: caller arrays of 2.
 * *hnorm (optional): sum_p |A_p| (1 + |z_p|) / (1 - |z_p|), a bound on the
 * l1 norm of h.  ABF_ERR_INVALID outside 2..5 or for NULL arrays.           */
abf_status abf1d_prefilter_host(int32_t n1, int32_t* npoles, double* z, double* A, double* hnorm);

/* Test hook for the failure path of the scans (no counterpart in the paper):
 * runs one line pass (direction v3) of the non-adaptive step with the CTAs of
 * its first band skipped, so the next band's look-back waits on flags that
 * nothing sets.  That wait is bounded: it gives up (about a second), sets
 * ABF_DEV_TIMEOUT in the plan's status word and the pass completes; the
 * context stays usable.  Every later band may wait out the limit too, so use
 * it on small plans.  d_g is left undefined.  Exact form only.              */
abf_status abf_debug_starved_lookback(abf_plan plan, void* d_g, void* d_ws, cudaStream_t stream);

/* Throughput probes behind the mesh's integer roofline (no counterpart in
 * the paper): kind 0 measures 32-bit integer multiply-adds per second, kind 1
 * the two-limb x 64-bit carry-chained multiply-accumulates per second (the
 * mesh's per-weight operation at order 2), both on eight independent chains
 * per thread over 8 CTAs of 256 threads per SM.  Synchronises the device;
 * allocates 32 KB for the duration of the call.                            */
abf_status abf_probe_alu(int32_t kind, double* ops_per_s);

/* Library version, for the bindings. */
int32_t abf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ABF_H */
