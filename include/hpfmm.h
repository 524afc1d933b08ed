/*
 * hpfmm.h -- C ABI of the half-plane Robin Laplace FMM (arXiv 2507.21913)
 * for NVIDIA GB300 (sm_103a).
 *
 * The library evaluates, for N points r_j = (x_j, y_j) with y_j > 0 and real
 * charges Q_j (Section 2.2, Eqs. potential1, 1.2, reactioncomp1,
 * reactioncomp2),
 *
 *   u(r_i) = sum_{j != i} Q_j (-1/2pi) ln|r_i - r_j|
 *          + sum_j        Q_j (+1/2pi) ln|r_i - r_j^im|,   r_j^im = (x_j, -y_j)
 *          + sum_j        Q_j [ I_0(x_i - x_j, y_i + y_j) + I_0(x_j - x_i, y_i + y_j) ]
 *
 * with I_n(x, y) = 1/(2 pi n!) int_0^inf e^{-lambda (y - i x)} lambda^n /
 * (lambda - kappa) d lambda (Eq. generalintegral; real kappa: the lambda path
 * passes below the pole, Eq. dzGreensfunimplossless), i.e. u = sum_j Q_j
 * G(r_i, r_j) for the Robin Green's function of Eq. ddGreensfunimp with
 * boundary condition dG/dy + kappa G = 0 on y = 0.  The sum is computed by the
 * FMM of Algorithms 1 and 2: one quadtree over the points whose mirror covers
 * the image sources, the classic log expansions for the free and image parts
 * and the paper's S2M / M2M / M2L / L2L / LE-evaluation operators for the
 * reaction parts (Eqs. MEcoefficients, metome, metoleimage, letole1,
 * truncatedLE).
 *
 * Conventions for every entry point
 *   - Pointers may be host or device memory (the library asks the CUDA
 *     runtime which); host buffers are staged through plan-owned device
 *     memory (allocated by the first such call), their copies on a
 *     plan-owned copy stream ordered against `stream` by events.  All work is
 *     ordered on `stream` (a cudaStream_t, NULL = legacy default stream):
 *     parts of a rebuild (reaction tables) and of a single-precision
 *     evaluation (the far-field passes, concurrent with the near field) run
 *     on plan-owned streams that are forked from `stream` and joined back
 *     into it with events, so the results are complete when `stream` reaches
 *     the call's end.  A plan's calls must not run concurrently with each
 *     other.
 *   - Outputs are in the caller's point order.  Complex values are stored as
 *     interleaved (re, im) doubles.
 *   - The caller owns every input and output buffer; a plan owns its tree,
 *     tables and workspace and never aliases caller memory after a call
 *     returns.
 *   - No exception crosses the ABI.  A non-OK status is returned
 *     synchronously; hpfmm_last_error() gives a one-line reason (per thread).
 *   - Device failures inside a kernel (bounded waits that gave up, bad sizes)
 *     are reported through the plan's status word by the next synchronising
 *     call (hpfmm_sync) rather than by faulting the GPU.
 */
#ifndef HPFMM_H
#define HPFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpfmm_plan hpfmm_plan; /* opaque */

typedef enum {
  HPFMM_OK = 0,
  HPFMM_EINVAL = 1,      /* invalid argument (y <= 0, non-finite, kappa or p out of range) */
  HPFMM_ENOMEM = 2,      /* device allocation failed */
  HPFMM_ECUDA = 3,       /* a CUDA runtime call failed */
  HPFMM_ETIMEOUT = 4,    /* a bounded device wait gave up */
  HPFMM_EUNSUPPORTED = 5 /* valid but outside what the library implements */
} hpfmm_status;

typedef enum {
  HPFMM_FP64 = 0,  /* every step in double precision (the plain path) */
  HPFMM_FP32 = 1,  /* P2P, M2L and expansions in single precision; translation
                      tables generated in double and rounded */
  HPFMM_MIXED = 2  /* as FP32, plus double precision for reaction P2P pairs
                      with y_i + y_j < tau_fp64 (close to the boundary) */
} hpfmm_precision;

typedef struct {
  hpfmm_precision prec; /* default HPFMM_FP64 */
  double tau_fp64;      /* MIXED only: boundary-distance threshold, default 0.05 */
  int levels;           /* 0: choose the uniform tree depth from leaf_size;
                           otherwise force the leaf level (1..15) */
  int subtree_levels;   /* 0: automatic; otherwise the depth (1..4) of the subtree
                           tiles of the fused upward / downward passes (one block per
                           subtree of 4^k leaves), clamped to what fits in shared memory */
  int m2l_mode;         /* free-space M2L of multi-RHS single-precision evaluations
                           (16 or more charge vectors): 0 the FP32 FMA kernel,
                           1 the tensor cores (tcgen05 kind::tf32, three-term split
                           products accumulated in tensor memory) */
  int adaptive;         /* 0: uniform tree (depth `levels`); 1: adaptive quadtree, in
                           which a box is split while it holds more than leaf_size
                           points, down to depth `levels` (0: automatic, at most 13).
                           Free-space M2L over same-level V-lists, near field over
                           the U-list extended by the W/X pairs (Section 3, the
                           paper's adaptive tree over targets and image sources).
                           Single and mixed precision, p <= 31; hpfmm_eval (one pass
                           set per charge vector), hpfmm_eval_adjoint, batched graphs
                           and hpfmm_update_points (hpfmm_eval_targets returns
                           HPFMM_EUNSUPPORTED for adaptive plans). */
  int async_update;     /* 0 (default): hpfmm_update_points waits for the device once,
                           after the tree build, and returns EINVAL / EUNSUPPORTED
                           for invalid points synchronously.  1: it does not wait;
                           the tree build writes the root square and the level
                           geometry on the device, where the evaluation kernels
                           read them, invalid points (non-finite, y <= 0) and an
                           out-of-range |kappa| * side are reported by the next
                           hpfmm_sync (HPFMM_EINVAL / HPFMM_EUNSUPPORTED), and the
                           outputs of an evaluation on such a tree are undefined
                           (finite or not; no memory outside the plan's buffers is
                           touched).  Uniform trees only (adaptive plans always
                           wait). */
  int reserved[1];      /* must be zero */
  double root_x0;       /* with root_side > 0: the root square of the tree is
                           [root_x0, root_x0 + root_side] x [0, root_side] instead of the
                           points' bounding square; it must contain every point
                           (EINVAL otherwise).  Used to cover separate targets
                           (hpfmm_eval_targets). */
  double root_side;
} hpfmm_options;

/* Fill *opt with the defaults. */
void hpfmm_default_options(hpfmm_options *opt);

/*
 * hpfmm_create -- build the tree and the translation tables for one point set
 * (Algorithm 1: images, tree over targets and image sources, tables).
 *   x, y       : n doubles each, host or device; y[i] > 0, all finite.
 *   n          : number of points, 1 <= n <= 2^31 - 1.
 *   kappa      : Robin parameter Z_eps = kappa_re + i kappa_im with
 *                kappa_re > 0, kappa_im >= 0 (Section 2.1); kappa_im == 0 is
 *                the lossless case.
 *   p          : expansion order, 1 <= p <= 40.
 *   leaf_size  : target mean number of points per leaf box, >= 1; the tree is
 *                uniform with depth round(log4(n / leaf_size)) clamped to
 *                [1, 12] unless opt->levels forces it.
 *   opt        : may be NULL (defaults).
 *   stream     : cudaStream_t for all device work of this call.
 *   out        : receives the plan.
 * The points are copied and sorted by Morton key; the plan keeps no pointer
 * to x or y.  Returns EUNSUPPORTED when |kappa| * sqrt(5) * (tree side) > 60,
 * the range in which the device evaluation of I_n is accurate to ~1e-13.
 */
hpfmm_status hpfmm_create(const double *x, const double *y, int64_t n, double kappa_re,
                          double kappa_im, int p, int leaf_size, const hpfmm_options *opt,
                          void *stream, hpfmm_plan **out);

/*
 * hpfmm_update_points -- rebuild the plan's tree and tables for a new set of
 * n points (same n as at creation, same kappa, p and options), reusing the
 * plan's device memory: validation, bounding square, Morton keys and sort,
 * leaf offsets and translation tables, as in hpfmm_create, without device
 * allocations after the first call (host coordinates are staged through a
 * plan-owned buffer, allocated by the first host-buffer call).  Without
 * async_update, returns EINVAL (synchronously) for invalid points, the plan
 * then holding no valid tree until a successful update, and the call waits
 * only until the bounding square is known on the device (its validity and
 * size reach the host through a pinned buffer); with async_update it does
 * not wait at all (see hpfmm_options).  The rest of the rebuild stays queued
 * on `stream`; the reaction tables are built on a plan-owned stream after
 * the tree build, which the evaluation joins before it reads them.
 */
hpfmm_status hpfmm_update_points(hpfmm_plan *plan, const double *x, const double *y,
                                 void *stream);

/*
 * hpfmm_eval -- u = G q for nrhs charge vectors on the plan's points
 * (Algorithm 2: free FMM + image FMM + reaction FMM for Phi_2^+ and Phi_2^-,
 * summed).
 *   q     : nrhs * n doubles, row r = charge vector r (caller order).
 *   nrhs  : >= 1.
 *   pot   : nrhs * n complex doubles (2 * nrhs * n doubles): u.
 *   grad  : NULL, or nrhs * n * 2 complex doubles: (du/dx_i, du/dy_i) per
 *           point (the field is minus this).
 * Stream-ordered; returns without synchronising unless host buffers are
 * involved (then the results are in host memory when it returns).
 */
hpfmm_status hpfmm_eval(hpfmm_plan *plan, const double *q, int nrhs, double *pot, double *grad,
                        void *stream);

/*
 * hpfmm_eval_adjoint -- gradient of a real functional L of u = G q with
 * respect to the charges and the positions of the plan's points (the
 * backward pass of hpfmm_eval for one charge vector).  The paper states the
 * kernel's symmetry G(r, r') = G(r', r) (Eq. greensfunsymm); with it the
 * transpose sums are forward sums with the charges Re g and Im g:
 *   dL/dq_j = Re u[Re g]_j + Im u[Im g]_j
 *   dL/dr_k = Re(conj(g_k) grad u[q]_k) + q_k (Re grad u[Re g]_k + Im grad u[Im g]_k)
 *   q      : n doubles, the charges of the forward evaluation (caller order);
 *            may be NULL when dxy is NULL.
 *   g      : n complex doubles (2n doubles), g_i = dL/dRe u_i + i dL/dIm u_i.
 *   grad_q : NULL, or the forward's grad output for q (n * 2 complex doubles);
 *            when NULL and dxy is wanted, one more evaluation computes it.
 *   dq     : NULL, or n doubles: dL/dq.
 *   dxy    : NULL, or n * 2 doubles: (dL/dx_k, dL/dy_k).
 * All arrays are device memory (EINVAL otherwise); at least one output.
 * Costs two evaluations (three without grad_q) and allocates a 20 n double
 * workspace in the plan on first use.  Stream-ordered.
 */
hpfmm_status hpfmm_eval_adjoint(hpfmm_plan *plan, const double *q, const double *g,
                                const double *grad_q, double *dq, double *dxy, void *stream);

/*
 * Batched evaluation of independent problems (one plan and one charge vector
 * each) as one CUDA graph.  The paper treats one problem at a time; this
 * entry point has no counterpart there: it issues the problems' evaluations
 * (hpfmm_eval's passes, unchanged) on nbranch parallel branches of one graph,
 * problems assigned to branches largest first, so that small problems share
 * the GPU.
 *   hpfmm_batch_create : plans[nprob] (distinct; the batch does not own them and
 *                        they must outlive it); nbranch = parallel branches
 *                        (0: min(nprob, 8)); creates the batch's streams.
 *   hpfmm_eval_batched : q[i] (n_i doubles), pot[i] (n_i complex), grad NULL or
 *                        grad[i] (n_i * 2 complex) -- device memory only, as in
 *                        hpfmm_eval.  The first call captures the graph; later
 *                        calls replay it while the pointers and the plans'
 *                        bounding squares are unchanged, else capture it again.
 *                        Ordered after earlier work on `stream`, and later work
 *                        on `stream` is ordered after it.  Plans with pass timing
 *                        on are rejected (EINVAL).  Calls on one batch must not
 *                        overlap, and the plans must not be evaluated elsewhere
 *                        meanwhile (they share the plans' workspaces).
 *   hpfmm_batch_captures : how many times the graph has been captured.
 *   hpfmm_batch_destroy  : waits for the batch's work and frees its streams.
 */
typedef struct hpfmm_batch hpfmm_batch;
hpfmm_status hpfmm_batch_create(hpfmm_plan *const *plans, int nprob, int nbranch,
                                hpfmm_batch **out);
hpfmm_status hpfmm_eval_batched(hpfmm_batch *batch, const double *const *q, double *const *pot,
                                double *const *grad, void *stream);
hpfmm_status hpfmm_batch_captures(const hpfmm_batch *batch, int64_t *captures);
hpfmm_status hpfmm_batch_destroy(hpfmm_batch *batch);

/*
 * hpfmm_autotune -- choose p, the leaf level and the subtree tile depth for
 * one point set by measurement (the paper fixes p from its error theorems and
 * does not tune the tree; this entry point has no counterpart there).
 *   x, y     : n device doubles (the points), n >= 64.
 *   prec     : HPFMM_FP64 / HPFMM_FP32 / HPFMM_MIXED.
 *   tol      : target relative L2 error, of the potential and of its gradient.
 *   nsample  : number of sampled targets (>= 8) for the error estimate.
 * A probe charge vector (a hash of the point index, uniform in [-1, 1)) is
 * evaluated by the FMM and, at every (n / nsample)-th point, by hpfmm_direct in
 * double precision; a configuration's error is the larger of the sampled
 * relative L2 errors of the potential and of the gradient.  For each leaf
 * level (the default level from n / 32 and one level either side) the
 * smallest even p (4..40) whose error meets tol is
 * taken and hpfmm_update_points + hpfmm_eval is timed with CUDA events; the
 * fastest wins (met = 1).  If no configuration meets tol, the most accurate
 * one seen is returned (met = 0).  The subtree depth (automatic or 1..4) is
 * then chosen by timing the winner.  Allocates and frees its own
 * device memory and synchronises the stream.  Use the result with
 * hpfmm_create(p, opt.levels = levels, opt.subtree_levels = subtree_levels).
 */
typedef struct {
  int p;
  int levels;
  int subtree_levels;
  int met;             /* 1 if est_rel_err <= tol */
  double mean_leaf;    /* n / 4^levels */
  double est_rel_err;  /* sampled relative L2 error of the chosen configuration */
  double ms_per_eval;  /* update_points + eval, potentials and gradients */
  int nsample;
} hpfmm_tuning;
hpfmm_status hpfmm_autotune(const double *x, const double *y, int64_t n, double kappa_re,
                            double kappa_im, int prec, double tol, int nsample, void *stream,
                            hpfmm_tuning *out);

/*
 * hpfmm_eval_targets -- u and its gradient at nt separate targets (the paper's
 * Example 2: field points on a mesh, including points on y = 0), from the
 * plan's sources with charges q (Algorithm 2 with the evaluation moved from
 * the sources to the targets: the far field from the local expansion of the
 * leaf containing the target, the near field -- free part, and image and
 * reaction parts next to y = 0 -- from the sources of the 3 x 3 neighbouring
 * leaves, summed in double precision).
 *   q      : n doubles, the sources' charges (caller order).
 *   xt, yt : nt doubles, finite, y_t >= 0, inside the plan's root square (create
 *            the plan with opt.root_x0 / root_side covering them); EINVAL otherwise.
 *   pot    : nt complex doubles; grad: NULL or nt x 2 complex doubles.
 * A target that coincides with a source skips that pair's free term.  All
 * arrays device memory.  Validates the targets with one synchronisation.
 */
hpfmm_status hpfmm_eval_targets(hpfmm_plan *plan, const double *q, const double *xt,
                                const double *yt, int64_t nt, double *pot, double *grad,
                                void *stream);

/* Release every device allocation of the plan (synchronises its stream). */
hpfmm_status hpfmm_destroy(hpfmm_plan *plan);

/*
 * hpfmm_direct -- O(N_t N_s) all-pairs evaluation of the same sum on the
 * device (no tree), in double precision.  Targets may differ from sources;
 * self_index[i] is the source index equal to target i (excluded from the
 * free part, Eq. 1.2) or -1, and may be NULL when targets are not sources.
 * Targets need y_t >= 0, sources y_s > 0.  grad may be NULL.
 */
hpfmm_status hpfmm_direct(const double *xs, const double *ys, const double *qs, int64_t ns,
                          const double *xt, const double *yt, const int64_t *self_index,
                          int64_t nt, double kappa_re, double kappa_im, double *pot,
                          double *grad, void *stream);

/* Plan geometry (host-side values). */
typedef struct {
  int64_t n;
  int levels;      /* leaf level H (boxes per side 2^H) */
  int p;
  int prec;
  double x0, side; /* bounding square [x0, x0 + side] x [0, side] */
  int64_t workspace_bytes;
} hpfmm_plan_info;
hpfmm_status hpfmm_get_info(const hpfmm_plan *plan, hpfmm_plan_info *info);

/*
 * hpfmm_get_adaptive_counts -- shape of an adaptive plan's tree (for checks):
 * boxes[l] and leaves[l], l = 0..maxlev (host arrays of maxlev + 1 entries,
 * zero beyond the tree), and in *depth (may be NULL) the deepest level that
 * has a box.  A box is split into its non-empty children while it holds more
 * than leaf_size points and its level is below opt.levels.  EINVAL for a
 * uniform plan.  Synchronises the stream.
 */
hpfmm_status hpfmm_get_adaptive_counts(const hpfmm_plan *plan, int maxlev, int64_t *boxes,
                                       int64_t *leaves, int *depth, void *stream);

/*
 * hpfmm_get_order -- copy the plan's Morton ordering (for checks): keys[k] is
 * the 60-bit key of the k-th point in tree order and perm[k] its index in the
 * caller's order.  Either pointer may be NULL; host or device memory.
 * Synchronises the stream.
 */
hpfmm_status hpfmm_get_order(const hpfmm_plan *plan, uint64_t *keys, int64_t *perm, void *stream);

/*
 * Pass timing.  hpfmm_set_timing(plan, 1) makes the plan record a CUDA event
 * pair around every pass it launches, on the stream that runs the pass (the
 * caller's stream or one of the plan's streams).  The passes, in the order
 * of their ids 0..9: tree build, tables, charge gather, P2M, M2M, free M2L,
 * mirror M2L, L2L, leaf evaluation = L2P + free-space near field (+ the image
 * and reaction near field in double precision), image and reaction near
 * field of the bottom-row leaves (single precision).
 * hpfmm_read_timing synchronises with that work and returns, per pass, the
 * device milliseconds recorded since the previous read (ms may be NULL) and the
 * number of kernels the plan has launched in that pass since creation
 * (launches may be NULL; counted whether or not timing is on).
 */
hpfmm_status hpfmm_set_timing(hpfmm_plan *plan, int enable);
hpfmm_status hpfmm_read_timing(hpfmm_plan *plan, double ms[10], int64_t launches[10]);

/*
 * The same records as a timeline: for each pass interval recorded since the
 * previous read (in recording order, at most cap of them), its pass id and
 * its begin and end in device milliseconds from the earliest recorded begin.
 * The passes run on several streams, so intervals overlap where passes run
 * concurrently; the gaps and the longest chain show the step's critical
 * path.  Synchronises with the recorded events and consumes the records as
 * hpfmm_read_timing does (read one or the other).  *count = the number of
 * intervals written.  EINVAL for a NULL plan or count, or NULL arrays with
 * cap > 0.
 */
hpfmm_status hpfmm_read_timeline(hpfmm_plan *plan, int cap, int *pass, double *begin_ms,
                                 double *end_ms, int *count);

/* Wait for the plan's outstanding work on `stream` and report any device-side
 * status (HPFMM_ETIMEOUT) recorded by its kernels. */
hpfmm_status hpfmm_sync(hpfmm_plan *plan, void *stream);

/*
 * hpfmm_tree_order_noalloc -- the tree ordering of hpfmm_get_order (sorted
 * 60-bit Morton keys and the permutation to the caller's order) computed
 * without any device allocation, for callers that cannot let a library
 * allocate device memory (a runtime that owns every device allocation, or a
 * process that must not grow its device memory use once it runs).  The paper
 * has no counterpart: this is a service entry point of the library.
 *   x, y   : n doubles each, device memory of the CURRENT device, y > 0,
 *            finite.
 *   n      : 1 <= n <= 65536 (larger n is rejected with HPFMM_EINVAL).
 *   levels : leaf level used to bucket the points, 1..8 (the result does not
 *            depend on it; leaves of any size are sorted on the device).
 *   keys   : n uint64, perm: n int64, device memory of the current device,
 *            written in tree order.
 * Pointers that are not device memory of the current device are rejected
 * with HPFMM_EINVAL.  All temporaries live in one static device array of
 * 2.5 MiB that every GPU holding the library keeps until the process exits.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress).  Every call reuses the same array: calls that
 * overlap on the GPU (several streams, several threads) race and must be
 * serialised by the caller.  The call reads the points' validity flag back
 * to the host, so it synchronises `stream` before it returns.
 */
hpfmm_status hpfmm_tree_order_noalloc(const double *x, const double *y, int64_t n, int levels,
                                      uint64_t *keys, int64_t *perm, void *stream);

/*
 * hpfmm_selftest_wait_timeout -- failure-path check of the library's bounded
 * device waits (no counterpart in the paper): launches one kernel whose
 * bulk-copy barrier can never complete, so its wait runs out of polls and the
 * kernel records a timeout in a status word instead of hanging.  Returns
 * HPFMM_ETIMEOUT when the timeout was reported (the expected outcome, after
 * about a second), HPFMM_OK if the wait somehow completed.  Synchronises.
 */
hpfmm_status hpfmm_selftest_wait_timeout(void *stream);

/*
 * hpfmm_selftest_tc_gemm -- check of the library's tensor-core building blocks
 * (no counterpart in the paper): one CTA computes D[128 x n] = A[128 x k] B^T
 * (B is n x k) with tcgen05 kind::tf32 MMAs accumulating in tensor memory,
 * in plain tf32 (split = 0) or as the three-term tf32 split product
 * hi*hi + hi*lo + lo*hi (split = 1).  All arrays row-major float, device
 * memory; 16 <= n <= 128 with n % 16 == 0, 8 <= k <= 64 with k % 8 == 0.
 * Returns ETIMEOUT if the MMA completion wait gave up.  Synchronises.
 */
hpfmm_status hpfmm_selftest_tc_gemm(const float *A, const float *B, float *D, int n, int k,
                                    int split, void *stream);

/*
 * hpfmm_measure_alu_peaks -- throughput of the arithmetic pipes that bound the
 * library's kernels, measured on the current device (no counterpart in the
 * paper; the denominators of the roofline fractions the benchmark reports):
 *   mufu_ops_per_s    special-function unit: lg2.approx.f32 + rcp.approx.f32,
 *                     the two SFU operations of a single-precision near-field
 *                     pair, counted as one operation each;
 *   ffma_flops_per_s  FP32 fused multiply-add, 2 flops each;
 *   dfma_flops_per_s  FP64 fused multiply-add, 2 flops each.
 * Each kernel runs 8 independent chains per thread on (multiprocessors x
 * resident blocks) blocks of 256 threads; the rate is the best of 5 timed
 * launches (CUDA events on `stream`).  *_mhz is the effective SM clock of that
 * launch (clock64 cycles / globaltimer ns of one block), *_per_clk_sm the
 * rate per clock and multiprocessor.  Changes no GPU setting.  Allocates 4 KB
 * of device memory for the duration of the call; synchronises `stream`.
 */
typedef struct {
  int sms;                       /* multiprocessors of the device */
  double mufu_ops_per_s, ffma_flops_per_s, dfma_flops_per_s;
  double mufu_mhz, ffma_mhz, dfma_mhz;
  double mufu_per_clk_sm, ffma_flops_per_clk_sm, dfma_flops_per_clk_sm;
} hpfmm_alu_peaks;
hpfmm_status hpfmm_measure_alu_peaks(hpfmm_alu_peaks *out, void *stream);

const char *hpfmm_status_string(hpfmm_status s);
const char *hpfmm_last_error(void);

/* Library version and build target, e.g. "hpfmm 0.1 sm_103a". */
const char *hpfmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HPFMM_H */
