/*
 * octmc — GB300-native (sm_103a) orthogonal-raster OCT/OCTA motion
 * correction: the joint registration objective, its per-A-scan displacement
 * gradient, and the multi-resolution L-BFGS solve around it.
 *
 * Method: Ploner et al., "Efficient and high accuracy 3-D OCT angiography
 * motion correction in pathology" (arXiv 2010.06931), Sec. 2.1-2.4.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Grid: w x h A-scans of d samples (Sec. 2.1).  0-based indices i (x,
 *    fast axis of the X-fast scan), j (y), k (depth), in pixels of the level.
 *  - Volumes: float32 [h][w][d], depth contiguous, both scans in the common
 *    frame (the Y-fast scan is NOT stored in its acquisition order).
 *  - En-face angiography A^V (Eq. 6): float32 [h][w].
 *  - Validity v^X: float32 [h] (one value per X-fast B-scan = row j);
 *    v^Y: float32 [w] (one value per Y-fast B-scan = column i)  (Sec. 2.2).
 *  - Sampling-time maps t^V: float64 [h][w], any monotone unit (they order
 *    the A-scans for the temporal regulariser and weight flyback steps).
 *  - Displacements D and gradients: float64 [2][3][h_l][w_l] =
 *    [volume X,Y][component dx,dy,dz][j][i] of level l (Sec. 2.1: one
 *    3-D displacement per A-scan and volume).
 *  - Objective (Eq. 1 with Eq. 9): f = eta*S^str + S^ang/eta + alpha*R + M.
 *    R sums, over each scan's time-ordered A-scans, the pseudo-Huber penalty
 *    of consecutive displacement differences (flyback steps weighted lower)
 *    times the level depth d, the per-A-scan scale of the data term that
 *    Eq. 6 also applies to the angio term.  The validity of Eq. 7 is
 *    resampled by the Hermite interpolant with zero node tangents, so
 *    0 <= delta <= delta_0 (Eq. 8).
 *  - Every call is ordered on the problem's CUDA stream; "device" pointers
 *    are CUDA global memory the caller owns; "host" pointers are ordinary
 *    memory.  Calls on one problem are not thread-safe.  An evaluation forks
 *    the mean-term sums onto an internal stream of the calling thread and
 *    joins them back before its regulariser kernel, so the caller sees
 *    plain stream order.
 *  - Return codes: 0 OK, 1 NOT_CONVERGED (soft: results are valid), negative
 *    = hard error (see OCTMC_ERR_*); no exception crosses this boundary.
 */
#ifndef OCTMC_H
#define OCTMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OCTMC_OK 0
#define OCTMC_NOT_CONVERGED 1
#define OCTMC_ERR_INVALID_ARG (-1)
#define OCTMC_ERR_OOM (-2)
#define OCTMC_ERR_CUDA (-3)
#define OCTMC_ERR_NONFINITE (-4)
#define OCTMC_ERR_TIMEOUT (-5)
#define OCTMC_ERR_UNSUPPORTED (-6)
#define OCTMC_ERR_SCRATCH_LIMIT (-7)

typedef enum { OCTMC_F32 = 0, OCTMC_BF16 = 1, OCTMC_F16 = 2 } octmc_dtype;
typedef enum { OCTMC_LOSS_PSEUDO_HUBER = 0, OCTMC_LOSS_SSD = 1 } octmc_loss;

typedef struct octmc_problem octmc_problem; /* opaque; owns all its device memory */

/* Problem description (Sec. 2.1 inputs plus solver settings). */
typedef struct {
    int w, h, d;          /* level-0 grid; each >= 1                                  */
    int storage;          /* octmc_dtype of the device copies of S^X, S^Y              */
    const float *sx, *sy; /* [h][w][d] structural volumes (required)                   */
    const float *ax, *ay; /* [h][w] en-face angiography, or both NULL (delta = 0)      */
    const float *vx, *vy; /* vx[h], vy[w] validity, or NULL (all B-scans valid)        */
    const double *tx, *ty;/* [h][w] sampling-time maps (required)                      */
    int inputs_on_device; /* 1: the pointers above are device memory, 0: host memory   */
    double alpha;         /* weight of the temporal regulariser R (default 0.1)        */
    double delta0;        /* default angio weight delta_0, Eq. 8 (default 0.5)         */
    double eps_h;         /* pseudo-Huber parameter of the data term, Eq. 4 (0.001)    */
    double eps_r;         /* pseudo-Huber parameter of R (default 0.01 px)             */
    double mu;            /* weight of M; <= 0 selects 1/(2 w_l h_l) per level          */
    int loss;             /* octmc_loss                                                */
    int levels;           /* pyramid levels, >= 1 (factor 2 each, Sec. 2.1)            */
    int lbfgs_m;          /* L-BFGS history length, 1..32 (default 8)                  */
    int max_iter;         /* L-BFGS iterations per level (default 5000)                */
    int max_ls;           /* objective evaluations per line search                     */
    double gtol;          /* stop when max|grad| <= gtol                               */
    double ftol;          /* stop after 3 iterations of relative decrease < ftol (1e-7) */
    void *stream;         /* cudaStream_t (NULL = the legacy default stream)           */
    int persistent_ascans;/* levels of at most this many A-scans are solved by one
                             persistent cooperative kernel (all iterations in one
                             launch, grid barriers between phases); 0: never
                             (default: on this GPU the graph-driven loop is faster
                             at every level size measured).  Problems run by the
                             server never use it.                                  */
} octmc_desc;

/* Per-level statistics of a solve. */
typedef struct {
    int level;            /* pyramid level solved                                      */
    int iters;            /* accepted L-BFGS iterations                                */
    int evals;            /* objective + gradient evaluations                          */
    int status;           /* 0 converged, 1 iteration cap, 2 line search exhausted,
                             3 a grid barrier of the persistent level kernel timed out */
    double f;             /* final objective                                           */
    double eta;           /* eta used on this level (Eq. 10)                           */
    double seconds;       /* wall time of the level                                    */
} octmc_stats;

/* Fills a description with the defaults named above (pointers NULL). */
void octmc_desc_defaults(octmc_desc *desc);

/* Creates a problem: validates the description, copies the inputs to the
 * device (converting the volumes to `storage` with round-to-nearest-even),
 * builds the factor-2 pyramid (Sec. 2.1; box mean, odd sizes repeat the
 * edge sample) and the time-ordered A-scan chains of each level.
 * The caller's buffers may be freed afterwards.  *out receives the problem.
 * Errors: INVALID_ARG (NULL required pointer, dims < 1, levels too deep for
 * the grid, unknown dtype/loss), OOM, CUDA, UNSUPPORTED (no sm_103a device). */
int octmc_create_problem(const octmc_desc *desc, octmc_problem **out);

/* Releases every device and host resource of the problem (NULL is a no-op). */
void octmc_destroy_problem(octmc_problem *p);

/* Grid size (w, h, d) of pyramid level `level` (0 = full resolution). */
int octmc_level_shape(const octmc_problem *p, int level, int *w, int *h, int *d);

/* Sets eta (Eq. 9) used by later evaluations of `level` (eta > 0, finite). */
int octmc_set_eta(octmc_problem *p, int level, double eta);

/* Eq. 10: eta = sqrt(S^ang_0.5(D0) / S^str_0.5(D0)) at the device field
 * disp0 (always with delta_0 = 0.5).  eta = 1 without angiography or when
 * either sum is zero or not finite.  Stores it for the level and returns it
 * in *eta_out (host). */
int octmc_compute_eta(octmc_problem *p, int level, const double *disp0_dev, double *eta_out);

/* Objective and gradient at the device field disp_dev of `level` (Eq. 1-10
 * with the regulariser and mean-term readings documented in the design
 * notes).  *f_host receives f (host, may be NULL); grad_dev (device, may be
 * NULL) receives df/dD in the displacement layout.  Uses the level's stored
 * eta (1 until set or computed).  Errors: INVALID_ARG, CUDA, NONFINITE
 * (f is NaN/Inf: the gradient is still written). */
int octmc_eval_objective_grad(octmc_problem *p, int level, const double *disp_dev, double *f_host,
                              double *grad_dev);

/* octmc_eval_objective_grad enqueued on `stream` (a cudaStream_t; NULL: the
 * problem's own stream) without waiting for it: the host is not
 * synchronised and no result comes back to the host.  terms_dev (device, may
 * be NULL) receives [S^str, S^ang, R, M, f, eta] as 6 doubles when the
 * evaluation completes in stream order; grad_dev as for the synchronous call.
 * Consecutive calls on one stream may reuse the problem's scratch buffers;
 * calls on one problem must not be issued on two streams at once.  A
 * non-finite f is not reported here (terms_dev holds it).  Errors:
 * INVALID_ARG, CUDA (a launch failed). */
int octmc_eval_objective_grad_async(octmc_problem *p, int level, const double *disp_dev, double *grad_dev,
                                    double *terms_dev, void *stream);

/* As octmc_eval_objective_grad, and terms_host[6] receives
 * [S^str, S^ang, R, M, f, eta] (Eq. 5, Eq. 6, R, M, f, eta). */
int octmc_eval_terms(octmc_problem *p, int level, const double *disp_dev, double *terms_host,
                     double *grad_dev);

/* Objectives (and gradients) of several independent problems evaluated
 * together, as octmc_eval_objective_grad does for one: one launch per
 * kernel for all of them (mean-term sums, data term per storage type,
 * regulariser), each problem with the blocks, partition and reduction order
 * of an evaluation of it alone, so every result equals the single call's.
 *   problems[k] (distinct), levels[k], disp_dev[k] (device field of that
 *   level), grad_dev[k] (device, may be NULL, or grad_dev itself NULL),
 *   f_host[k] (host, may be NULL) receives f.
 * Each problem uses its level's stored eta.  The call first waits for the
 * problems' own streams, then orders all work on the stream of problems[0]
 * and returns when it is done.  count is 1..4096.
 * Errors: INVALID_ARG, CUDA, NONFINITE (some f not finite; all outputs are
 * written). */
int octmc_eval_batch(octmc_problem *const *problems, int count, const int *levels, const double *const *disp_dev,
                     double *const *grad_dev, double *f_host);

/* L-BFGS solve of one level (Sec. 2.1) from the device field disp_inout
 * (overwritten with the result).  eta is first computed from the initial
 * field (Eq. 10).  Returns OK, NOT_CONVERGED (iteration cap) or an error;
 * st (host, may be NULL) receives the statistics. */
int octmc_solve_level(octmc_problem *p, int level, double *disp_inout_dev, octmc_stats *st);

/* Full coarse-to-fine solve (Sec. 2.1): zero displacements at the coarsest
 * level, solve, prolong (x2 values, centre-aligned bilinear), ... down to
 * level 0.  disp_out_dev receives the level-0 field; st (host, may be
 * NULL) receives `levels` entries ordered coarse to fine. */
int octmc_solve_full(octmc_problem *p, double *disp_out_dev, octmc_stats *st);

/* Prolongs a displacement field of level `level` (device) to level-1
 * (device): every component doubled, bilinear at (i - 1/2)/2 on the coarse
 * grid with clamped coordinates. */
int octmc_prolong(octmc_problem *p, int level, const double *coarse_dev, double *fine_dev);

/* Final resampling and merging at level 0 (Sec. 2.1 last paragraphs,
 * Sec. 2.5) for the level-0 device field disp0_dev ([2][3][h][w] float64):
 *   corrected_x / corrected_y (device float32 [h][w][d]): each scan resampled
 *     at p_ijk + d^V_ij with the objective's interpolator;
 *   weights (device float32 [2][h][w]): normalised per-A-scan merge weights.
 *     The sampling density of scan V is the map of the positions
 *     (i + dx^V, j + dy^V) (clamped into the grid) splatted bilinearly with
 *     weight 1, read back bilinearly at A-scan (i, j)'s own position; the raw
 *     weight is exp(-beta * max(0, density - 1)), weights below tau are set
 *     to 0, the pair is normalised to sum 1, and where both were clipped the
 *     scan with the larger raw weight is kept alone;
 *   merged (device float32 [h][w][d]): wX C^X + wY C^Y;
 *   angio (device float32 [h][w]): en-face angiography images resampled at
 *     the displaced transverse positions, merged with the clipped raw
 *     weights times the resampled validity (Eq. 7), 0 where both are 0.
 * Any output may be NULL.  The density map is accumulated in 64-bit
 * fixed point (2^-32 units), so the result is deterministic.  Typical
 * beta = 2, tau = 0.05.  Errors: INVALID_ARG (beta < 0, tau outside [0, 1]),
 * OOM (first call allocates 16 w h bytes of density maps kept by the
 * problem), CUDA. */
int octmc_merge(octmc_problem *p, const double *disp0_dev, double beta, double tau, float *merged,
                float *corrected_x, float *corrected_y, float *weights, float *angio);

/* ---------------------------------------------------------------------
 * Rough axial prealignment (stage 1 of Sec. 2.1: "only estimates axial
 * displacements and tilt at B-scan granularity").  Parameters of a level
 * with w x h A-scans, device float64 [aX(h), tX(h), aY(w), tY(w)]: the
 * X-fast B-scan j (a row) moves A-scan (i, j) axially by
 * aX_j + tX_j (i - (w-1)/2), the Y-fast B-scan i (a column) by
 * aY_i + tY_i (j - (h-1)/2); transverse displacements are 0.  Objective:
 * S_0^str + alpha R + M + T (Eq. 1), the structural term alone (delta_0 = 0,
 * eta = 1) on the induced field, and the tilt term T, which fixes the three
 * deformations of the common frame the data cannot see (a common x tilt,
 * y tilt and x y twist), each weighted like M for the same displacement
 * energy: T = 2 w vx sX^2 / h + 2 h vy sY^2 / w + 2 w h vx vy sT^2 / nT^2,
 * vx = (w^2-1)/12, vy = (h^2-1)/12, sX = sum tX, sY = sum tY,
 * sT = sum_j tX_j (j - cy) + sum_i tY_i (i - cx), nT = h vy + w vx (the
 * paper defers T's form to earlier work).  The solver is the 3-D solve's L-BFGS
 * with the same line search, limits and history length.
 * --------------------------------------------------------------------- */

/* The field [2][3][h][w] (device) induced by the parameters of `level`. */
int octmc_prealign_disp(octmc_problem *p, int level, const double *prm_dev, double *disp_dev);

/* Stage-1 objective at prm_dev: *f_host (host, may be NULL) and its
 * gradient grad_prm_dev (device, 2 (w + h) values, may be NULL).
 * Errors: INVALID_ARG, CUDA, NONFINITE. */
int octmc_prealign_eval(octmc_problem *p, int level, const double *prm_dev, double *f_host,
                        double *grad_prm_dev);

/* L-BFGS solve of the stage-1 objective of one level from prm_inout_dev
 * (overwritten).  Returns OK, NOT_CONVERGED (iteration cap) or an error. */
int octmc_prealign_level(octmc_problem *p, int level, double *prm_inout_dev, octmc_stats *st);

/* Coarse-to-fine stage-1 solve from zero parameters: between levels fine
 * B-scan b takes the coarse parameters at (b - 1/2)/2 (clamped, linear),
 * offsets doubled, tilts kept.  prm_out_dev (device, 2 (w + h) of level 0)
 * receives the level-0 parameters, disp0_out_dev (device, may be NULL) the
 * induced level-0 field; st (host, may be NULL) `levels` entries, coarse
 * to fine. */
int octmc_prealign_full(octmc_problem *p, double *prm_out_dev, double *disp0_out_dev, octmc_stats *st);

/* ---------------------------------------------------------------------
 * Angiography preprocessing of one scan (inputs of the objective).
 * Volumes are device float32 [h][w][d] (depth contiguous) on the common
 * grid; fast_axis 0: X-fast scan, B-scans are the rows j (h of them);
 * fast_axis 1: Y-fast scan, B-scans are the columns i (w of them).
 * stream: a cudaStream_t (NULL: the legacy default stream).  Both calls
 * synchronise the stream before returning; scratch comes from the
 * stream-ordered allocator and is released before returning.
 * --------------------------------------------------------------------- */

/* Saccade validity (Sec. 2.2): m_b = mean of the OCTA volume over B-scan b;
 * B-scan b is saturated if m_b > mu + 3 sigma (mean and population standard
 * deviation of the m_b); v_dev[b] (device, one float per B-scan) is 0 if b
 * or a B-scan within 2 of it is saturated, else 1.  means_dev (device, may
 * be NULL) receives the m_b (float64).  Errors: INVALID_ARG, CUDA. */
int octmc_saccade_validity(const float *octa_dev, int w, int h, int d, int fast_axis, float *v_dev,
                           double *means_dev, void *stream);

/* En-face OCTA image (Sec. 2.3): 3x3x3 median of the OCTA volume, then the
 * 3rd smallest of 15 samples along the fast axis, then along the slow axis
 * (edges replicated); the q_lo / q_hi quantiles (linear interpolation between
 * order statistics) of the filtered voxels of the valid B-scans (all if none
 * is valid) map to 0 / 1 and voxels below `thresh` form the lateral-contrast
 * mask; voxels whose OCT value exceeds t_oct (NaN: the mean OCT value over
 * the valid B-scans) form the OCT mask.  enface_dev [h][w] receives the depth
 * mean of the OCTA voxels in both masks (0 where none), minus the median of
 * its B-scan, with invalid B-scans (v_dev == 0) replaced by the nearest valid
 * one (lower index on a tie).  filtered_dev (device [h][w][d], may be NULL)
 * receives the rank-filtered volume; info_host (may be NULL) receives
 * [q_lo quantile, q_hi quantile, t_oct, voxels in both masks].  The paper
 * uses q_lo = 0.05, q_hi = 0.95, thresh = 0.1.  Inputs must be finite.
 * Errors: INVALID_ARG, UNSUPPORTED (more than 4096 A-scans per B-scan, h > 65535), OOM,
 * CUDA. */
int octmc_enface(const float *octa_dev, const float *oct_dev, int w, int h, int d, int fast_axis,
                 const float *v_dev, double q_lo, double q_hi, double thresh, double t_oct, float *enface_dev,
                 float *filtered_dev, double *info_host, void *stream);

/* Copies pyramid data of `level` to device buffers (any may be NULL):
 * sx/sy as float32 [h][w][d], ax/ay [h][w], vx[h], vy[w]. */
int octmc_level_data(const octmc_problem *p, int level, float *sx, float *sy, float *ax, float *ay,
                     float *vx, float *vy);

/* ---------------------------------------------------------------------
 * Stand-alone L-BFGS (Sec. 2.1) over n float64 device values: the compact
 * representation of the inverse Hessian with gamma = s'y / y'y of the latest
 * pair; pairs with s'y <= 1e-12 y'y are rejected.  The pairs, every product
 * with them and every sum are float64 (fixed reduction order, so results are
 * reproducible); an empty history gives exactly -g.  m is 1..32.
 * --------------------------------------------------------------------- */
typedef struct octmc_lbfgs octmc_lbfgs;

int octmc_lbfgs_create(int64_t n, int m, void *stream, octmc_lbfgs **out);
void octmc_lbfgs_destroy(octmc_lbfgs *h);
/* Appends the pair (s, y) (device).  Returns 0 if stored, 1 if rejected. */
int octmc_lbfgs_push(octmc_lbfgs *h, const double *s_dev, const double *y_dev);
/* dir_dev = -H g_dev for the stored pairs; *gtd_host (may be NULL) = g'dir. */
int octmc_lbfgs_direction(octmc_lbfgs *h, const double *g_dev, double *dir_dev, double *gtd_host);
/* Drops every stored pair. */
int octmc_lbfgs_reset(octmc_lbfgs *h);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of independent full solves (Sec. 2.1 per
 * request).  Requests wait in a FIFO queue and are admitted while a slot is
 * free and their estimated device memory (octmc_estimate_bytes) fits the
 * budget; once admitted their problem lives on the device.  Each
 * octmc_server_step runs ONE batched objective evaluation for every admitted
 * request (each at its own pyramid level, iteration and line-search trial;
 * one launch per kernel for all of them) and then each request's L-BFGS
 * bookkeeping.  A request's result does not depend on the other requests in
 * the batch: its kernels use the same partition and reduction order as a
 * solve of it alone (octmc_solve_full).  All work is on the server's stream.
 * --------------------------------------------------------------------- */
typedef struct octmc_server octmc_server;

#define OCTMC_REQ_UNKNOWN (-1)
#define OCTMC_REQ_QUEUED 0
#define OCTMC_REQ_RUNNING 1
#define OCTMC_REQ_DONE 2

/* Device bytes a problem with this description needs while it is solved
 * (volumes of every level, 16-bit conversion temporaries, workspace, L-BFGS
 * history, result); -1 for an invalid size. */
int64_t octmc_estimate_bytes(const octmc_desc *desc);

/* budget_bytes: device memory the admitted requests may use together;
 * max_slots: requests solved together at most; stream: cudaStream_t. */
int octmc_server_create(int64_t budget_bytes, int max_slots, void *stream, octmc_server **out);
void octmc_server_destroy(octmc_server *s);

/* Queues a full solve of `desc` (its stream field is ignored).  The arrays
 * the description points to must stay valid until the request has been
 * admitted (state RUNNING or DONE).  *ticket identifies the request.
 * Errors: INVALID_ARG; OOM if the request can never fit the budget. */
int octmc_server_submit(octmc_server *s, const octmc_desc *desc, int64_t *ticket);

/* Admits what fits, then one batched evaluation step for all admitted
 * requests.  *active / *queued (may be NULL) receive the counts after the
 * step.  A request whose admission fails is DONE with its error code. */
int octmc_server_step(octmc_server *s, int *active, int *queued);

/* *state = OCTMC_REQ_* of the request; nothing else happens. */
int octmc_server_state(const octmc_server *s, int64_t ticket, int *state);

/* *state = OCTMC_REQ_*.  When DONE: the level-0 displacement field is copied
 * to disp_out_dev (device, 6*w*h float64, may be NULL), up to max_stats
 * per-level statistics (coarse to fine) to stats, the request's return code
 * to *req_rc, and the request's memory is released (the ticket is then
 * unknown). */
int octmc_server_poll(octmc_server *s, int64_t ticket, int *state, double *disp_out_dev, octmc_stats *stats,
                      int max_stats, int *req_rc);

/* ---------------------------------------------------------------------
 * Kernel timing: when enabled, every evaluation records CUDA events on the
 * problem's stream around the data-term kernel (resampling, loss and
 * per-A-scan gradient) and adds the elapsed time once the evaluation has
 * synchronised.  Enabling resets the totals.
 * --------------------------------------------------------------------- */
int octmc_profile_enable(octmc_problem *p, int enable);
/* Total milliseconds and number of timed data-term launches so far. */
int octmc_profile_read(octmc_problem *p, double *total_ms, long long *launches);

/* ---------------------------------------------------------------------
 * Data term without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (code inside a
 * memory-pool or allocator callback, frameworks that own all device memory,
 * paths where allocating after start-up is forbidden).  It evaluates
 * S^str = sum (1 - delta) sum_k L(R_ijk) and S^ang = sum delta d L(R_ij(A))
 * (Eq. 5, 6) of one grid and eta*S^str + S^ang/eta's gradient with respect
 * to the displacements, using the same kernel as the other entry points.
 *   sx, sy: device float32 [h][w][d] with d a multiple of 4 (>= 4), 16-byte
 *           aligned;
 *   ax, ay: device [h][w] or both NULL; vx[h], vy[w]: device or NULL;
 *   disp: device float64 [2][3][h][w];
 *   grad_out: device float64 [2][3][h][w] or NULL (data-term gradient);
 *   sums_out: device float64 [2] receives S^str, S^ang.
 * Its scratch is one file-scope device array of 8 MiB (+2.4 KiB), held by
 * every GPU that loads the library until the process exits; it fits grids
 * of at most 262,144 A-scans (w*h); larger grids return
 * OCTMC_ERR_SCRATCH_LIMIT, and w*h*d/4 must stay below 2^32.  Each call
 * looks up the array's device address (cudaGetSymbolAddress) for the
 * current device; the first lookup on a device may load the module there,
 * so make the first call before any stream capture.  eta, delta0 and eps_h
 * must be finite.  Every call shares the array and
 * leaves its contents behind: calls that overlap on the GPU (other streams,
 * other threads, same device) race and give wrong results.  Asynchronous on
 * `stream`; errors: INVALID_ARG, SCRATCH_LIMIT, CUDA.
 * --------------------------------------------------------------------- */
int octmc_data_term_static(const float *sx, const float *sy, const float *ax, const float *ay,
                           const float *vx, const float *vy, int w, int h, int d, const double *disp,
                           double eta, double delta0, double eps_h, int loss, double *grad_out,
                           double *sums_out, void *stream);

/* Self-test of the bounded grid barrier that the persistent level kernel
 * (persistent_ascans > 0) waits at between its phases: a cooperative grid of
 * one block per SM waits once for `extra` (0 or 1) more blocks than it has.
 * extra = 0: the barrier completes (OK).  extra = 1: it cannot complete, so
 * every block's wait runs out after its iteration or time limit (about 2 s)
 * and the call returns TIMEOUT; nothing traps and the context stays usable.
 * Errors: INVALID_ARG, OOM, CUDA. */
int octmc_barrier_selftest(int extra);

/* Human-readable name of a return code. */
const char *octmc_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* OCTMC_H */
