/*
 * mra.h -- C ABI of the GB300 separated-operator apply library (libmra.so).
 *
 * The library applies an integral operator whose kernel is written as a sum of
 * Gaussians (the Poisson kernel 1/r or the bound-state Helmholtz kernel
 * exp(-mu r)/r) to a function held as order-k Legendre scaling-function
 * coefficients on an adaptive 3-D tree, as described in Harrison et al.,
 * "MADNESS: A Multiresolution, Adaptive Numerical Environment for Scientific
 * Simulation" (arXiv 1507.01888), Sec. 2.1-2.3.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Cell [-L, L]^3.  Level n has 2^n boxes per dimension of width h_n = 2L/2^n
 *    (Sec. 2.1 maps the domain to [0,1]; the library scales it to the cell).
 *  - Box key (uint64): level << 57 | x << 38 | y << 19 | z, 0 <= x,y,z < 2^n,
 *    n <= 19.  Trees hold their keys sorted ascending, without duplicates.
 *  - Coefficients: k^3 doubles per box, s[ix][iy][iz] row-major (ix slowest),
 *    in the basis phi^n_{b,i}(x) = h_n^{-1/2} phi_i((x+L)/h_n - b),
 *    phi_i(x) = sqrt(2i+1) P_i(2x-1) (Sec. 2.1, eq. scalingfunc).
 *  - Every call returns an int status: MRA_OK (0) or a negative MRA_ERR_*.
 *    mra_last_error() returns a thread-local message for the last failure.
 *    Nothing throws across this interface.
 *  - Host arrays passed in are read during the call only; the library keeps
 *    no caller host pointer.  Device buffers (tree views, workspace) are owned
 *    by the caller: size queries come first, the caller allocates.  Opaque
 *    handles (mra_operator) are owned by the library and freed with
 *    mra_operator_free.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered; a call that must learn a size on the
 *    host (mra_project, mra_apply) synchronises that stream before returning.
 */
#ifndef MRA_H
#define MRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define MRA_OK 0
#define MRA_ERR_ARG (-1)      /* invalid argument (null pointer, bad size or order) */
#define MRA_ERR_CAPACITY (-2) /* a caller buffer is too small; the required size is reported */
#define MRA_ERR_CUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define MRA_ERR_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define MRA_ERR_NUMERIC (-5)  /* a non-finite value was produced */
#define MRA_ERR_UNSUPPORTED (-6) /* valid, but outside what this path supports (e.g. a split order above 16) */

/* ---- enumerations --------------------------------------------------------- */
#define MRA_POISSON 0 /* K(r) = 1/r                          (Sec. 2.3) */
#define MRA_BSH 1     /* K(r) = exp(-mu r)/r, mu = sqrt(-2E)  (Sec. 3.2, eq. bshkernel
                         without its 1/(4 pi), which the caller applies) */

#define MRA_PREC_FP64 0       /* all arithmetic in FP64 */
#define MRA_PREC_SPLIT_BF16 1 /* mode products as split-BF16 tcgen05 MMAs: every operand is
                                 split into `pieces` BF16 pieces and the piece products p + q <
                                 pieces are accumulated in FP32 in tensor memory.  Sums over
                                 Gaussian terms: the source-stationary kernel (even k 4..10) sums
                                 up to opts.join terms in the tensor-memory accumulator, then adds
                                 them into each (source, displacement) sum in plain or compensated
                                 FP32 (opts.sums), stored as FP32 and summed per destination in
                                 FP32 pairs (error-free TwoSum additions, about 48 bits) formed
                                 into FP64; the destination-stationary kernel keeps compensated FP32
                                 sums per destination, formed into FP64 at the end.  Operator
                                 blocks, fit, norms and screen stay FP64.  Measured error: 1.2e-7
                                 to 1.8e-7 relative L2 against MRA_PREC_FP64 with 3 pieces; use
                                 MRA_PREC_FP64 for thresholds below that */

#define MRA_SCREEN_NONE 0 /* keep every term */
#define MRA_SCREEN_NORM 1 /* keep a term iff |c| ||Rx|| ||Ry|| ||Rz|| ||s|| >= tau */
#define MRA_SCREEN_LEARNED 2 /* the norm screen, then also skip a kept term when the learned
                                 model predicts log10 ||term|| + delta < log10 tau */

#define MRA_STENCIL_SHELLS 0  /* shells of |l|_inf = 0,1,..,max_disp, stop at the first empty shell */
#define MRA_STENCIL_NEAREST 1 /* all 27 displacements with |l|_inf <= 1 */

#define MRA_MAX_LEVEL 19
#define MRA_MAX_K 16
#define MRA_MAX_NS_K 20 /* largest order 2k of a non-standard-form operator (k <= 10); orders
                           above MRA_MAX_K are applied with MRA_PREC_FP64 only */
#define MRA_MAX_TERMS 128
#define MRA_NOALLOC_MAX_BOXES (1 << 20) /* largest tree mra_norm_noalloc accepts */
#define MRA_MAX_FUNCS 2048 /* functions in one mra_apply_batched call */
#define MRA_MLP_PARAMS 4555 /* floats of a learned-screen model (see mra_mlp_init) */

/* ---- data types ----------------------------------------------------------- */

/* f(x) = sum_g coef[g] exp(-expnt[g] |x - c_g|^2); host arrays of length n. */
typedef struct {
  int n;
  const double *coef, *expnt, *cx, *cy, *cz;
} mra_gauss_sum;

/* A tree on the device: n boxes (keys sorted ascending) with k^3 doubles each.
 * cap is the number of boxes the two buffers can hold. */
typedef struct {
  int64_t n;
  int64_t cap;
  uint64_t *keys;  /* device, cap entries */
  double *coeffs;  /* device, cap * k^3 entries */
  int k;
  double L;
} mra_tree_view;

typedef struct mra_operator mra_operator; /* opaque */

typedef struct {
  int precision;  /* MRA_PREC_* */
  int pieces;     /* split pieces per operand for MRA_PREC_SPLIT_BF16 (2 or 3) */
  int screen;     /* MRA_SCREEN_* */
  double tau;     /* screen threshold (ignored for MRA_SCREEN_NONE) */
  int stencil;    /* MRA_STENCIL_* */
  int max_disp;   /* largest |l|_inf for MRA_STENCIL_SHELLS (<= the operator's max_disp) */
  const float *mlp; /* MRA_SCREEN_LEARNED: device model, MRA_MLP_PARAMS floats */
  double delta;     /* MRA_SCREEN_LEARNED: safety margin in log10 units */
  int tile_variant; /* MRA_PREC_SPLIT_BF16 tile shape: 0 = four 128-row tiles per CTA (one CTA
                       per SM); 1 (k >= 4) = two tiles per CTA (two CTAs per SM); 2 (k = 4 to
                       10) = one tile per CTA (four CTAs per SM); others are taken as 0 */
  const double *delta_level; /* MRA_SCREEN_LEARNED, optional (NULL = delta at every level): host
                                array of MRA_MAX_LEVEL + 1 margins, one per source level, read
                                during the call; +inf keeps every term of that level */
  uint64_t dest_lo, dest_hi; /* destination partition (owner computes): only destinations whose
                                key lies in [dest_lo, dest_hi) are computed and written, with the
                                screen's shell decisions of the whole apply; dest_hi = 0 keeps all.
                                mra_apply only (not batched, not the non-standard form) */
  int split_kernel; /* MRA_PREC_SPLIT_BF16: MRA_SPLIT_AUTO (0) runs the source-stationary kernel
                       where it applies (even k from 4 to 10, records with |l|_inf <= 2) and the
                       destination-stationary one elsewhere; MRA_SPLIT_DEST (1) always the
                       destination-stationary one (tile_variant picks its shape) */
  int join;  /* source-stationary kernel: consecutive terms of a record group that the tile's
                records keep alike (the same records keep both) are summed in the tensor-memory
                accumulator, up to `join` of them (1..8), before one flush adds them into the record
                sums.  0: 2 in tiles of one source (k = 10) and 1 in tiles of several, whose results
                then do not depend on which sources share a tile (batched or partitioned applies
                equal the single ones bit for bit); a value >= 1 applies to every tile.  More terms
                per flush cost accuracy (the accumulator truncates) */
  int sums;  /* source-stationary kernel, each record's sum over terms: MRA_SUMS_PLAIN (0, an FP32
                sum; a ninth warp then issues stage 3) or MRA_SUMS_COMPENSATED (1, FP32 sum + Kahan
                correction: more accurate, more registers, eight warps) */
  int ahead; /* source-stationary kernel: block copies run this many terms ahead (1..4; 0 = 2) */
} mra_apply_opts;

#define MRA_SPLIT_AUTO 0
#define MRA_SPLIT_DEST 1
#define MRA_SUMS_PLAIN 0
#define MRA_SUMS_COMPENSATED 1

typedef struct {
  int64_t n_in;               /* source boxes */
  int64_t n_out;              /* destination boxes written */
  int64_t pairs;              /* (source, displacement) pairs with at least one kept term */
  int64_t terms_kept;         /* (source, displacement, Gaussian term) triples computed */
  int64_t terms_screened;     /* triples dropped by the screen inside the displacement set */
  int64_t terms_issued;       /* triples the kernel evaluated (kept + tile padding) */
  int64_t sources_truncated;  /* sources whose last allowed shell still kept terms */
  double skipped_bound;       /* sum of the screen bounds of dropped triples, or an upper bound of
                                 it: a bound the screen's FP32 log2 filter decided enters as
                                 2^(its FP32 log2 + 2^-8), at most 0.4% above it */
  double kernel_ms;           /* device time of the apply kernel and the kernels around it that its
                                 result needs (CUDA events on `stream`) */
  int64_t terms_learned_skipped; /* triples the norm screen kept and the learned screen dropped */
  double learned_skipped_bound;  /* sum of the norm-screen bounds of those triples */
  double algo_flops;  /* algorithmic flops of the kept triples: 6 k^4 + k^3 each, k the order
                         of the operator that applied them (k or 2k in the non-standard form) */
  int64_t level_sources[MRA_MAX_LEVEL + 1];    /* source boxes per level */
  int64_t level_terms_kept[MRA_MAX_LEVEL + 1]; /* kept triples per source level */
  int32_t kernel;     /* the apply kernel that ran: MRA_KERNEL_F64, MRA_KERNEL_SPLIT_DEST or
                         MRA_KERNEL_SPLIT_SRC (kernel_ms covers it with its work-list and
                         summation kernels); for the non-standard form, that of its last apply */
  double main_kernel_ms; /* device time of that kernel alone (CUDA events on `stream` around its
                            launch; equal to kernel_ms where the apply runs one kernel; summed
                            over the applies of the non-standard form) */
  int64_t mma_passes; /* source-stationary kernel: its passes (source tile, l_x, l_y, window of
                         three l_z, term), each one set of stage-1, 2 and 3 MMAs; 0 otherwise */
} mra_apply_stats;

#define MRA_KERNEL_F64 0        /* FP64 destination-stationary kernel */
#define MRA_KERNEL_SPLIT_DEST 1 /* split-BF16 destination-stationary tensor-core kernel */
#define MRA_KERNEL_SPLIT_SRC 2  /* split-BF16 source-stationary tensor-core kernel */

typedef struct {
  double diff_norm;  /* || test - ref ||_2 over the union of boxes */
  double ref_norm;   /* || ref ||_2 */
  double test_norm;  /* || test ||_2 */
  double rel_l2;     /* diff_norm / ref_norm */
  double max_box_rel;/* max over common boxes of ||test_b - ref_b|| / ||ref_b|| */
  int64_t n_common;  /* boxes present in both trees */
  int64_t n_only_test, n_only_ref;
  /* per level n = 0..MRA_MAX_LEVEL: || test - ref ||_2 and || ref ||_2 over the boxes of level n
     (boxes present in only one tree count with the other side as zero) and the number of boxes
     of level n in ref */
  double level_diff_norm[MRA_MAX_LEVEL + 1];
  double level_ref_norm[MRA_MAX_LEVEL + 1];
  int64_t level_ref_boxes[MRA_MAX_LEVEL + 1];
} mra_compare_result;

/* ---- calls ---------------------------------------------------------------- */

/* Number of kernels the library has launched in this process so far (every launch of every
 * entry point, counted on the host when it is issued; library routines the calls use, such as
 * the CUB sorts and scans, are not counted).  Take the difference around a region of calls. */
long long mra_launch_count(void);

/* Device memory the library keeps for reuse: the scratch of the calls that allocate it
 * themselves (projection, norms and comparisons, reconstruction, truncation, products, the
 * non-standard applies) comes from a stream-ordered pool per device that holds on to freed
 * memory between calls.  This returns the pool's unused memory to the driver.  Memory of
 * allocations still in flight on a stream is not affected. */
int mra_release_memory(void);

/* Test hook for the failure path: the next MRA_PREC_SPLIT_BF16 apply in this process has one
 * CTA (the one that takes the first tile) skip the block copies of its first term, so that the kernel's bounded waits on them
 * run out (about two seconds each); that apply returns MRA_ERR_TIMEOUT with the device context
 * intact, and later calls run normally.  One-shot; nothing else is changed. */
int mra_debug_inject_stall(void);

/* The checking build (libmra_debug.so, compiled with MRA_DEBUG): the hot kernels' gather and
 * scatter indices (records, sources, operator blocks) are checked against their ranges; an
 * index out of range is replaced by 0, so the access stays in bounds, and the first failing
 * source line is kept.  mra_debug_status synchronises `stream`, writes that line (0: no
 * failure since the last call) to *line and clears it; the release build always writes 0.
 * mra_debug_selftest sends one out-of-range index through the check (a test of the checking
 * path itself; a no-op in the release build). */
int mra_debug_status(int *line, void *stream);
int mra_debug_selftest(void *stream);

/* FP64 throughput of the current device, measured (the paper has no counterpart; this is the
 * denominator of the FP64 apply's roofline).  Two probes over the whole device (eight CTAs of
 * 256 threads per SM), each timed with CUDA events as the best of three launches of about
 * seconds/8 each after a calibration launch: *dfma_tflops, independent DFMA chains (the
 * instructions apply_f64 uses); *dmma_tflops, mma.sync m16n8k16 FP64 warp MMAs.  Either
 * pointer may be NULL.  Takes about `seconds` (0 < seconds <= 60) of GPU time on `stream` and
 * synchronises it; allocates nothing. */
int mra_measure_fp64_peak(double seconds, double *dfma_tflops, double *dmma_tflops, void *stream);

/* Thread-local description of the last error (never NULL). */
const char *mra_last_error(void);

/* Library version string. */
const char *mra_version(void);

/* Size in bytes of the ABI structure named `name` ("mra_gauss_sum", "mra_tree_view",
 * "mra_apply_opts", "mra_apply_stats", "mra_compare_result"), or -1 for another name.  Lets a
 * binding check its copies of the structures' layouts without a GPU. */
int64_t mra_abi_sizeof(const char *name);

/* Project f onto the scaling functions (Sec. 2.1, eq. projection):
 * s^n_b = int f phi^n_b, computed per box from exact 1-D Gaussian integrals.
 * uniform_level >= 0: every box of that level.  uniform_level < 0: adaptive
 * refinement (Sec. 2.1): every box of level init_level-1 is a parent; a
 * parent's 8 children are projected exactly and compared with the parent's
 * own projection expressed on the children (two-scale relation, Sec. 2.2);
 * if the Frobenius norm of the difference is <= thresh, or the children are
 * at max_level, the children become leaves, else each child becomes a parent.
 * out: device buffers with out->cap boxes; on success out->n, out->k, out->L
 * are set and the keys are sorted.  MRA_ERR_CAPACITY if out->cap is too small
 * (out->n then holds the required count).  Temporary device memory for the
 * refinement is allocated and freed on `stream` inside the call. */
int mra_project(const mra_gauss_sum *f, int k, double L, double thresh, int init_level,
                int max_level, int uniform_level, mra_tree_view *out, void *stream);

/* Build the separated operator (Sec. 2.3): the Gaussian fit of the kernel and
 * the 1-D operator blocks.
 * Fit: trapezoid rule of K(r) = (2/sqrt pi) int exp(-r^2 e^{2s} - mu^2 e^{-2s}/4 + s) ds
 * (mu = 0 gives the 1/r identity of Sec. 2.3) with M terms,
 *   c_m = (2/sqrt pi) h exp(s_m - mu^2 e^{-2 s_m}/4), t_m = e^{2 s_m}, s_m = s_lo + m h,
 * where (h, s_lo) minimise the maximum relative error on 3000 log-spaced r
 * in [r_lo, r_hi] over the grid h = 0.05..1.20 (step 0.01), s_lo = -25..3
 * (step 0.25); ties go to the smaller h.  r_hi <= 0 selects 2L, shortened to
 * ln(1/fit_eps)/mu for MRA_BSH.
 * Blocks (Toeplitz, Sec. 2.2): for every level n in [min_level, max_level],
 * term m < M and 1-D displacement |l| <= min(max_disp, 2^n - 1),
 *   R^n_{m,l}[i][j] = h_n int_0^1 int_0^1 phi_i(u) exp(-t_m h_n^2 (u - v + l)^2) phi_j(v) du dv,
 * which maps the source box b to the target box b + l, and its Frobenius norm.
 * *op receives a handle owning the device tables; free with mra_operator_free. */
int mra_operator_create(int kernel, double mu, int M, double fit_eps, double r_lo, double r_hi,
                        int k, double L, int min_level, int max_level, int max_disp,
                        mra_operator **op, void *stream);

/* The same call under the name of the block generator it runs (identical arguments, result and
 * errors): the Gaussian fit and every block R^n_{m,l} of the operator. */
int mra_operator_blocks(int kernel, double mu, int M, double fit_eps, double r_lo, double r_hi,
                        int k, double L, int min_level, int max_level, int max_disp,
                        mra_operator **op, void *stream);

/* The BSH operator refitted in place for a new mu (an iteration whose energy changed): the
 * Gaussian fit is searched again; when it lands on the same grid point (h, s_lo) the exponents
 * t_m, and so every block, are unchanged and only c_m and the c_m-scaled tensor-core pieces are
 * recomputed (*blocks_reused = 1), otherwise the blocks are computed again (0).  The result is
 * the operator mra_operator_create would make for mu.  Non-standard-form operators built from
 * op must be created again (refitting one of them is refused).  After an error the operator
 * may be half updated: free it. */
int mra_operator_refit(mra_operator *op, double mu, int *blocks_reused, void *stream);

/* Copy the fit out of an operator (host arrays of length M; any may be NULL). */
int mra_operator_fit(const mra_operator *op, double *c, double *t, double *h, double *s_lo,
                     double *max_rel_err);

/* Shape of an operator: k, M, levels and the largest displacement. */
int mra_operator_info(const mra_operator *op, int *k, int *M, int *min_level, int *max_level,
                      int *max_disp, double *L);

/* Copy one block R^n_{m,l} (k*k doubles, row i, column j) and its Frobenius norm to the host. */
int mra_operator_block(const mra_operator *op, int level, int m, int l, double *R, double *norm);

int mra_operator_free(mra_operator *op);

/* Device workspace (bytes) that mra_apply needs for this input and options. */
int mra_apply_workspace_size(const mra_operator *op, const mra_tree_view *in,
                             const mra_apply_opts *opts, size_t *bytes);

/* Apply the separated operator to `in` (Sec. 2.3), leaf level by leaf level:
 * for every source box b (level n), every displacement l in D(b) with b + l in
 * the cell, and every term m kept by the screen,
 *   r_{n,b+l} += c_m (s_b x_1 R^n_{m,lx} x_2 R^n_{m,ly} x_3 R^n_{m,lz}),
 * the three k x k mode products of the separated representation.
 * D(b): MRA_STENCIL_NEAREST -> |l|_inf <= 1; MRA_STENCIL_SHELLS -> shells
 * |l|_inf = 0, 1, ..., opts->max_disp, stopping after the first shell in which
 * no term is kept.  Screen MRA_SCREEN_NORM keeps a term iff
 *   |c_m| * ||R_x||_F * ||R_y||_F * ||R_z||_F * ||s_b||_F >= tau
 * (that product, in that order, bounds the term's norm).
 * Results stay at the source's level; every destination box is computed by
 * gathering its sources after a sort on the destination key, so each output
 * box is written exactly once (no atomics).  out: device buffers; out->n
 * receives the number of destination boxes, keys sorted ascending.
 * workspace: device buffer of at least mra_apply_workspace_size bytes.
 * stats may be NULL; when given, the call also waits for the apply kernel so
 * that stats->kernel_ms holds its device time.  Synchronises `stream` twice to
 * learn the record and output counts; MRA_ERR_CAPACITY (with out->n =
 * required) if out->cap is too small, before the apply kernel runs. */
int mra_apply(const mra_operator *op, const mra_tree_view *in, const mra_apply_opts *opts,
              mra_tree_view *out, void *workspace, size_t workspace_bytes,
              mra_apply_stats *stats, void *stream);

/* Learned screen (a 4 -> 64 -> 64 -> 1 tanh network in FP32, MRA_MLP_PARAMS floats on
 * the device).  It predicts log10 of a term's norm ||c_m (R_x x R_y x R_z) s_b||_F from the
 * features (level n, |l|_2, log10 t_m, log10 ||s_b||_F); MRA_SCREEN_LEARNED drops a term
 * that passed the norm screen when prediction + delta < log10 tau.  The paper has no
 * counterpart (its screen is the norm estimate of Sec. 2.2); the norm screen remains the
 * fallback and a bound on what the learned one may drop (learned_skipped_bound).
 * Parameter layout: W1[64][4], b1[64], W2[64][64], b2[64], W3[64], b3, x_mean[4], x_std[4],
 * y_mean, y_std; inputs are standardised by (x_mean, x_std), the output is scaled by
 * (y_std, y_mean). */

/* mra_apply on a tree in HOST memory: in->keys and in->coeffs, out->keys and out->coeffs are
 * host pointers (page-locked memory gives the full copy rate; pageable memory works but the
 * copies then block the calling thread).  The library copies the tree to the device, runs the
 * same apply as mra_apply (same kernels, same result bit for bit), copies the result boxes
 * into out (out->cap boxes at most) and synchronises the stream before returning; its device
 * scratch comes from the library's memory pool (see mra_release_memory).  When the result has
 * more than out->cap boxes nothing is copied, out->n receives the count and MRA_ERR_CAPACITY
 * is returned.  Every host<->device copy of the apply is inside this one call, which is what
 * an end-to-end measurement times. */
int mra_apply_host(const mra_operator *op, const mra_tree_view *in, const mra_apply_opts *opts,
                   mra_tree_view *out, mra_apply_stats *stats, void *stream);

/* Log training data from a plain apply: run the screen of mra_apply with `opts` (its
 * precision is ignored), draw about max_terms of the kept terms with a counter-based
 * hash of (seed, record, term) and write, for each, the features (device float[4]) and
 * log10 of the term's true norm in FP64 (device float).  *n_logged <= max_terms.
 * workspace: at least mra_apply_workspace_size bytes. */
int mra_log_terms(const mra_operator *op, const mra_tree_view *in, const mra_apply_opts *opts,
                  int64_t max_terms, uint64_t seed, float *features, float *log_norms,
                  int64_t *n_logged, void *workspace, size_t workspace_bytes, void *stream);

/* Initialise a model: uniform(+-sqrt(6/(fan_in+fan_out))) weights from a counter-based
 * generator of `seed`, zero biases, identity standardisation. */
int mra_mlp_init(float *params, uint64_t seed, void *stream);

/* Set the model's standardisation (mean and standard deviation of each feature and of
 * the target) from n logged rows (device arrays). */
int mra_mlp_standardize(float *params, const float *features, const float *targets, int64_t n,
                        void *stream);

/* Predictions (log10 term norms) for n rows of features; all device arrays. */
int mra_mlp_forward(const float *params, const float *features, int64_t n, float *out, void *stream);

/* Workspace bytes of mra_mlp_grad for n rows, or of mra_mlp_train for batches of n rows. */
int mra_mlp_workspace_size(int64_t n, size_t *bytes);

/* Full-batch gradient (device float[MRA_MLP_PARAMS], the trainable first 4545 entries
 * written) of the mean squared error between the standardised output and the
 * standardised targets, and that loss (host).  Deterministic. */
int mra_mlp_grad(const float *params, const float *features, const float *targets, int64_t n,
                 float *grad, double *loss, void *workspace, size_t workspace_bytes, void *stream);

/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, rate lr) on minibatches of
 * `batch` rows drawn with replacement by a counter-based generator of (seed, step).
 * adam_state: device float[2*MRA_MLP_PARAMS], zero before the first step; step0 = number
 * of steps already taken with this state.  *final_loss (host, may be NULL) = loss of the
 * last minibatch.  workspace: mra_mlp_workspace_size(batch) bytes. */
int mra_mlp_train(float *params, float *adam_state, const float *features, const float *targets,
                  int64_t n, int batch, int steps, int step0, float lr, uint64_t seed,
                  double *final_loss, void *workspace, size_t workspace_bytes, void *stream);

/* Apply one operator to nfunc functions in one pass: every kernel of mra_apply runs once
 * over all of them (the tensor-core tiles may mix functions, which share the operator's
 * blocks).  in: one tree view holding the functions' boxes back to back, function f at
 * [in_offsets[f], in_offsets[f+1]) (host array of nfunc+1, in_offsets[0] = 0,
 * in_offsets[nfunc] = in->n), each function's keys sorted.  out: one tree view; on return
 * function f's destination boxes are [out_offsets[f], out_offsets[f+1]) (host array of
 * nfunc+1), keys sorted within each function.  Levels above 15 are not supported here
 * (MRA_ERR_UNSUPPORTED); nfunc <= MRA_MAX_FUNCS.  Same workspace size query as mra_apply
 * with in; same statistics, summed over the functions.  The paper applies each function
 * separately; batching is this library's. */
int mra_apply_batched(const mra_operator *op, int nfunc, const mra_tree_view *in, const int64_t *in_offsets,
                      const mra_apply_opts *opts, mra_tree_view *out, int64_t *out_offsets, void *workspace,
                      size_t workspace_bytes, mra_apply_stats *stats, void *stream);

/* ---- Non-standard form (Sec. 2.2).  With P^{n+1} = P^n + Q^n the level-N operator is
 * T^N = T^{n0} + sum_{n=n0}^{N-1} (A^n + B^n + C^n), A^n = Q^n T Q^n, B^n = Q^n T P^n,
 * C^n = P^n T Q^n, whose blocks decay with the displacement (A as r^(-2k-1), B and C as
 * r^(-k-1)).  On level n's 2k basis (a box's children's coefficients side by side,
 * index (c, i) = c k + i per dimension) the level-(n+1) operator has the blocks
 *     R2k^n_{m,l}[(ci,i)][(cj,j)] = R^{n+1}_{m, 2l+ci-cj}[i][j].
 *
 * mra_operator_ns_create: the 2k-basis operator of levels op.min_level .. op.max_level-1
 * with displacements |l| <= max_disp, assembled on the device from op's blocks (op needs
 * max_disp >= 2 max_disp + 1 for that); its own norms, and its BF16 pieces when 2k <=
 * MRA_MAX_K.  2k <= MRA_MAX_NS_K; orders above MRA_MAX_K are applied with MRA_PREC_FP64 only
 * (a split request returns MRA_ERR_UNSUPPORTED).  Caller frees it with mra_operator_free. */
int mra_operator_ns_create(const mra_operator *op, int max_disp, mra_operator **ns_op, void *stream);

/* Workspace bytes of mra_apply_ns (device memory the caller provides, 256-byte aligned). */
int mra_apply_ns_workspace_size(const mra_operator *op, const mra_operator *ns_op, const mra_tree_view *in,
                                int n0, const mra_apply_opts *opts, size_t *bytes);

/* Non-standard form apply on a uniform tree.  in: every box of one level N (1..10) in key
 * order (keys sorted: x slowest), k^3 coefficients each; op: the operator (order k, levels
 * n0..N, max_disp >= 2^n0 - 1); ns_op: mra_operator_ns_create(op, ...).  Steps: compress
 * (s^n = filter of the children tensor S^n, n = N-1 .. n0); T^{n0} s^{n0} with every
 * displacement of level n0; for n = n0 .. N-1, Y^n = T2k^n S^n and Z^n = T^n s^n with
 * opts' stencil and screen (each an mra_apply on level n's boxes, in opts' precision),
 * and the children of every box b get U^{x3} (r^n_b - Z^n_b) + Y^n_b as r^{n+1}.  out:
 * the level-N result, same keys as in (cap >= in->n, else MRA_ERR_CAPACITY with out->n
 * the size needed).  opts.screen: NONE or NORM.  With every displacement the result equals
 * mra_apply's level-N result with every displacement.  stats: summed over the applies;
 * kernel_ms is the apply kernels' time only.  Synchronises the stream. */
int mra_apply_ns(const mra_operator *op, const mra_operator *ns_op, const mra_tree_view *in, int n0,
                 const mra_apply_opts *opts, mra_tree_view *out, void *workspace, size_t workspace_bytes,
                 mra_apply_stats *stats, void *stream);

/* Non-standard form apply on an adaptive tree.  in: the leaves of a complete octree (every
 * interior node has its eight children; keys sorted and unique), every leaf deeper than n0.
 * Sources of level n are the interior nodes (S = the children's coefficients, s = their
 * filter); the result tree starts with every box of level n0 (T^{n0} s^{n0}, every
 * displacement) and at each level n refines the nodes that level's applies (T2k^n on S,
 * T^n on s, opts' stencil and screen) reach: their children get U^{x3} (r_p - Z_p) + Y_p.
 * out: the result's leaves in key order (boxes of several levels, disjoint); if out->cap is
 * too small, MRA_ERR_CAPACITY with out->n the number needed.  A leaf of level n enters
 * through T^n, so with every displacement the result is, as a function, mra_apply's
 * leaf-level result with every displacement.  Allocates its temporaries on the stream
 * (cudaMallocAsync) and releases them before returning; synchronises the stream. */
int mra_apply_ns_tree(const mra_operator *op, const mra_operator *ns_op, const mra_tree_view *in, int n0,
                      const mra_apply_opts *opts, mra_tree_view *out, mra_apply_stats *stats, void *stream);

/* Reconstruct (sum-down, Sec. 2.2): boxes of any levels, keys sorted and unique, a box and
 * boxes below it both allowed (as mra_apply returns them: every destination at its source's
 * level), representing f = sum_b f_b; out: disjoint leaves holding the same function, keys
 * sorted.  Every box with input boxes below it, and every box on the path down to them, passes
 * its accumulated coefficients to its eight children through the two-scale relation; the
 * others are the leaves.  k <= MRA_MAX_K / 2.  Capacity as mra_apply_ns_tree; temporaries
 * stream-ordered; synchronises the stream. */
int mra_reconstruct(const mra_tree_view *in, mra_tree_view *out, void *stream);

/* Truncate (the refinement test of Sec. 2.1 run backwards): on disjoint leaves (keys sorted and
 * unique), from the deepest level up, eight sibling leaves whose detail d = S - U^{x3} s
 * (S their coefficients as one (2k)^3 tensor, s = its filter, the parent's coefficients) has
 * ||d||_F <= thresh are replaced by the parent holding s; a parent made so can merge again.
 * out: the remaining leaves, keys sorted (capacity as mra_reconstruct).  *err2 (host, may be
 * NULL): sum of ||d||^2 over the merges = the squared L2 change (d is orthogonal to the
 * parent's space).  Temporaries stream-ordered; synchronises the stream. */
int mra_truncate(const mra_tree_view *in, double thresh, mra_tree_view *out, double *err2, void *stream);

/* Product of two functions held on trees of disjoint leaves (keys sorted and unique; same k
 * and L).  Both are first summed down to their common refinement (each tree's leaves plus zero
 * boxes at the other's keys, through mra_reconstruct); then, per leaf, the values at the k
 * Gauss-Legendre points of each dimension (the third representation of Sec. 2.1) are
 * multiplied and transformed back: s_ab = h^{-3/2} (V^T W)^{x3} [(V^{x3} s_a)(V^{x3} s_b)],
 * V[q][i] = phi_i(x_q), W = diag(w_q) -- the product interpolated at the points.  out: the
 * common leaves (capacity as mra_reconstruct).  k <= MRA_MAX_K / 2.  Synchronises. */
int mra_multiply(const mra_tree_view *a, const mra_tree_view *b, mra_tree_view *out, void *stream);

/* Inner product <a, b> = integral of a b, the coefficient dot product over the two trees'
 * common leaves (orthonormal basis); deterministic reduction, *result on the host. */
int mra_inner(const mra_tree_view *a, const mra_tree_view *b, double *result, void *stream);

/* Multiply a function by a constant in place: every coefficient of tree->n boxes times alpha
 * (the basis is linear, so the coefficients of alpha f are alpha times those of f, Sec. 2.1).
 * The bound-state Helmholtz iteration of Sec. 3.2 uses it for the Green's function factor
 * -2 * 1/(4 pi) and for normalising psi.  Stream-ordered, no synchronisation; alpha finite. */
int mra_scale(mra_tree_view *tree, double alpha, void *stream);

/* ---- graph-captured apply --------------------------------------------------------------
 * An apply (nfunc == 1: as mra_apply; nfunc > 1: as mra_apply_batched, in_offsets and
 * out_offsets as there) recorded once as a CUDA graph and replayed with one launch.  Create
 * runs the apply once (its result is in `out` on return), learns its sizes (records after the
 * screen, destination boxes) and records the whole sequence -- norms, screen, sorts, the apply
 * kernel -- in a fixed-size mode without host synchronisation.  A replay reads in->keys and
 * in->coeffs and writes out->keys and out->coeffs at the addresses given here, so the caller
 * may change the input coefficients between replays (same in->n).  The workspace stays owned
 * by the graph until mra_apply_graph_free.  Every replay checks on the device that its record
 * and destination counts equal the recorded ones; mra_apply_graph_status synchronises the
 * stream, returns MRA_ERR_CAPACITY if any replay since the last call needed other sizes (its
 * output is then not valid: create the graph again), MRA_ERR_TIMEOUT if a tensor-core wait
 * gave up, and clears the record.  Statistics are not gathered by replays. */
typedef struct mra_apply_graph mra_apply_graph; /* opaque */
int mra_apply_graph_create(const mra_operator *op, int nfunc, const mra_tree_view *in, const int64_t *in_offsets,
                           const mra_apply_opts *opts, mra_tree_view *out, int64_t *out_offsets, void *workspace,
                           size_t workspace_bytes, mra_apply_graph **graph, void *stream);
int mra_apply_graph_launch(mra_apply_graph *graph, void *stream);
int mra_apply_graph_status(mra_apply_graph *graph, void *stream);
/* Destination boxes of the recorded apply and the library kernels one replay launches. */
int mra_apply_graph_info(const mra_apply_graph *graph, int64_t *n_out, long long *kernels_per_launch);
int mra_apply_graph_free(mra_apply_graph *graph);

/* Norm of a function on a tree (the L2 norm the worked example of Sec. 3.1 prints, next to
 * eq. gaussian, for the projected Gaussian).  The scaling functions are orthonormal (Sec. 2.1,
 * eq. scalingfunc), so the L2 norm of f restricted to a box is the Frobenius norm of the box's
 * coefficient tensor and ||f||_2^2 is the sum of their squares over disjoint boxes.  Writes the
 * per-box norms (device array of tree->n doubles, may be NULL) and the total
 * sqrt(sum_b ||s_b||_F^2) (host double, may be NULL); with boxes that overlap (a box and boxes
 * below it, as mra_apply returns them) the total is the coefficient norm, not ||f||_2.
 * Deterministic reduction; synchronises `stream`. */
int mra_norm(const mra_tree_view *tree, double *per_box, double *total, void *stream);

/* mra_norm without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code
 * whose device memory is owned entirely by another allocator (a framework's
 * caching allocator, or an application with a fixed memory budget), where a
 * cudaMalloc would fail or fragment that pool, and latency-critical loops that
 * cannot afford the device-wide synchronisation cudaMalloc/cudaFree may cause.
 * Same results as mra_norm (per-box norms into the caller's device array
 * per_box, may be NULL; total into the host double, may be NULL).
 * Scratch is one fixed array of MRA_NOALLOC_MAX_BOXES + 32 doubles (8 MiB) in
 * the library's device memory.  It is resident on a device from the first call
 * there (the library's device code, and the array with it, is loaded into a
 * context on first use) until the process exits; trees with more boxes are
 * rejected with MRA_ERR_CAPACITY before any GPU work.  Every call looks up the
 * array's address in the current device's context (cudaGetSymbolAddress); the
 * first call on a device loads the code there, so make it before any stream
 * capture.  All calls share the array and nothing carries
 * over between calls (every slot read is written earlier in the same call), but
 * calls that overlap on the GPU (e.g. on two streams) race on it.  The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Synchronises `stream`. */
int mra_norm_noalloc(const mra_tree_view *tree, double *per_box, double *total, void *stream);

/* Relative L2 error of `test` against `ref` (the error measure the apply's accuracy is stated
 * in: || test - ref ||_2 / || ref ||_2, also per level).  Both trees have the same k; boxes are
 * matched by key and a box present in one tree only counts in full (the other side as zero).
 * By the orthonormality of the basis (Sec. 2.1, eq. scalingfunc) coefficient differences are
 * function differences, so on trees of the same boxes diff_norm is the L2 norm of the difference
 * of the two functions.  Host result; synchronises `stream`. */
int mra_compare(const mra_tree_view *test, const mra_tree_view *ref, mra_compare_result *res,
                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MRA_H */
