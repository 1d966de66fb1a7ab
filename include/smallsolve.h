/*
 * smallsolve.h -- C ABI of the batched small structured-solve library
 * (CUDA, sm_103a).
 *
 * The operations are the three case studies of "Program Generation for Linear
 * Algebra Using Multiple Layers of DSLs" (Spampinato, Fabregat-Traver,
 * Pueschel, Bientinesi), Fig. 2 caption:
 *   potrf_upper:  X^T X = A           A SPD, X upper triangular   (Fig. 2a)
 *   trlyap_l:     L X + X L^T = S     L lower, S and X symmetric  (Fig. 2b)
 *   trsyl_lu:     L X + X U = C       L lower, U upper            (Fig. 2c)
 * all in double precision (the "Preliminary performance results" paragraph),
 * here for many independent small instances per call.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.  Every pointer argument whose name starts with d_ is a DEVICE
 * pointer.  The caller owns all memory; the library allocates nothing on the
 * solve path and never synchronises the stream.  Pointer arrays (d_A, d_X, ...)
 * are device arrays of `batch` device pointers; size arrays (d_n, d_ld*) are
 * device arrays of `batch` ints.
 *
 * Layout.  Instance b is column-major: element (i, j) of operand M sits at
 * d_M[b][i + j * d_ldm[b]], 0 <= i, j < d_n[b], with d_ldm[b] >= max(1, d_n[b]).
 *
 * Triangles.  Only the structurally meaningful triangle of an input is read:
 * A upper, L lower, U upper, S lower.  Only the upper triangle of the Cholesky
 * X and the lower triangle of the Lyapunov X are written; the other strict
 * triangle of X is left untouched.  The Sylvester X is written in full.
 * X may alias the right-hand side (X == A, X == C or X == S per instance with
 * the same leading dimension) in SS_MODE_FP64, SS_MODE_DF and the *_RAW modes; it must not
 * overlap anything else.  The *_REFINED modes read the original right-hand
 * side at every refinement step, so they need X separate from it (as
 * mixed-precision LAPACK drivers take B and X separately); an aliased
 * instance gets info = SS_INFO_ALIASED and is left untouched.
 *
 * Sizes.  0 <= d_n[b] <= max_n <= SS_MAX_N.  max_n is a host-side bound used to
 * size the launch; an instance whose device-side n violates it is skipped and
 * gets info = SS_INFO_BAD_SIZE.  n = 0 is an empty instance (info = 0).
 *
 * Modes (`mode`).  SS_MODE_FP64 computes in FP64 throughout.  The *_REFINED
 * modes solve in low precision (the update products in TF32 or BF16 on the
 * tensor cores with FP32 accumulation, or in FP32 on the CUDA cores; diagonal
 * blocks, square roots and divisions stay FP64) and then apply FP64 iterative
 * refinement until the relative correction falls below SS_REFINE_TOL or
 * SS_REFINE_MAXIT steps ran.  The *_RAW modes stop after the low-precision
 * solve.  Refined and raw modes need workspace (see ss_workspace_size).
 *
 * SS_MODE_DF: the warp-specialised pipeline with its block updates in
 * double-float arithmetic (each FP64 operand split into two floats, about 48
 * significant bits; error-free products and sums on the FP32 pipe).
 * trsyl_lu, trlyap_l, trsyl_rect: T = C - sum L X - sum X U and the
 * diagonal-block recurrences in double-float; the divisors l_ii + u_jj and
 * their reciprocals are computed in FP64; X is rounded to FP64.  potrf_upper,
 * posv_upper (factor stage): T = A - sum X^T X in double-float; the diagonal
 * blocks (square roots, pivots, panel solves) stay FP64; posv_upper's
 * triangular solves likewise.  No refinement.  Workspace: FP64's plus 24
 * bytes per instance, and the double-float copies the update warps stage
 * from (split once per instance): for trsyl_lu, trlyap_l and trsyl_rect of
 * L, U and X (24 bytes per max_n^2 per instance in the ss_workspace_size
 * bound), for potrf_upper and posv_upper of X (8 bytes per max_n^2); an
 * instance without room gets SS_INFO_NO_WORK.
 * Accuracy is that of FP64 up to the split's 2^-47 relative representation
 * error per operand.
 *
 * Magnitude.  The problems are plain double precision, so SS_MODE_DF and the
 * refined modes, which compute in FP32 arithmetic, rescale an instance by
 * powers of two where its data needs it (exact in binary floating point):
 * L and U by 2^a and C by 2^c (X then carries 2^(c-a)), moving the largest
 * entries of the operator and of the right-hand side to [1, 2) unless they
 * already lie in [2^-12, 2^13); a Cholesky A by 4^s (X by 2^s) unless its
 * largest entry lies in [2^-40, 2^41); for the SPD solve also B.  Data of any
 * FP64 magnitude is thus solved to the same accuracy; entries more than
 * 2^126 below the largest of their operand count as zero (a perturbation
 * below 2^-126 of the operand's norm).  In SS_MODE_DF the largest entries of
 * a Sylvester / Lyapunov instance are found by the solve's first pass over
 * it (which also splits L and U) and an instance outside the band is solved
 * by a second, rescaled launch; a Cholesky A is checked as the
 * factorisation reads it, and an instance outside the band is factored again
 * rescaled (as is, after a scan, every instance factored in place, X == A).
 * A Sylvester / Lyapunov instance whose rescaled solution reaches 2^60 (a
 * solution at least 2^60 times larger than its data) or holds Inf / NaN has
 * left the double-float range: a last launch of the group solves it again in
 * SS_MODE_FP64 from its right-hand side, or, when X overwrote that
 * right-hand side (X == C or X == S), sets info = SS_INFO_RANGE.  In the
 * refined modes such an instance ends as a refinement that did not converge
 * (info n + 1).
 *
 * SS_MODE_AUTO solves each size bin in the (mode, cfg) pair given by
 * ss_set_auto_table (the autotuner's or the learned selector's choice among
 * FP64, SS_MODE_DF and the refined modes, all of which meet the same
 * accuracy); bins the
 * table leaves unset run in SS_MODE_FP64 with the default configuration, and
 * `cfg` is ignored.
 *
 * Configurations (`cfg`).  cfg >= 0 selects a kernel configuration by id
 * (0 <= cfg < ss_config_count(op, mode)); cfg = SS_CFG_TABLE uses the per-size
 * table set with ss_set_config_table (the autotuner's or the learned
 * selector's choice), falling back to the built-in default for sizes the table
 * leaves at -1; cfg = SS_CFG_DEFAULT uses the built-in default.
 *
 * Return value.  0 on success; -k if argument k (1-based) is invalid, checked
 * on the host before anything is launched; SS_ERR_CUDA if a launch failed.
 * Per-instance numerical outcomes go to d_info[b] (written on the stream):
 *   0                  success;
 *   k > 0  (potrf)     leading minor k is not positive (pivot k-1, 0-based,
 *                      was <= 0 or NaN); columns >= k-1 of X are undefined;
 *   1      (trsyl, trlyap) some divisor l_ii + u_jj (l_ii + l_jj) has
 *                      magnitude <= n * DBL_EPSILON * max diagonal magnitude,
 *                      or is NaN; X is computed anyway and may hold Inf/NaN;
 *   n + 1  (refined modes) refinement did not reach SS_REFINE_TOL within
 *                      SS_REFINE_MAXIT steps; X holds the last iterate;
 *   SS_INFO_BAD_SIZE   d_n[b] < 0 or d_n[b] > max_n; X untouched;
 *   SS_INFO_NO_WORK    the workspace was too small for this instance;
 *   SS_INFO_ALIASED    (refined modes) X aliases the right-hand side; X untouched;
 *   SS_INFO_RANGE      (SS_MODE_DF, trsyl / trlyap / trsyl_rect, X == C or
 *                      X == S) the solution left the double-float range (see
 *                      Magnitude); X is undefined: solve again in SS_MODE_FP64.
 *   SS_INFO_TIMEOUT    (refined modes, tensor-memory configurations) the
 *                      bounded wait for the tensor cores ran out; X is
 *                      undefined, and that CTA took no further instances
 *                      (the others finish the batch).  Not expected in
 *                      normal operation.
 *
 * Streams.  `stream` is a cudaStream_t (NULL: the legacy default stream).
 * Every call is asynchronous with respect to the host.  When a call uses
 * several (mode, cfg) launch groups (SS_CFG_TABLE, SS_MODE_AUTO), groups after
 * the first run on the library's auxiliary streams (three per device, created
 * on first use), forked from `stream` after the pre-pass and joined back
 * before the call returns, so their persistent kernels overlap; the whole call
 * stays ordered on `stream` and can be captured into a CUDA graph.
 */
#ifndef SMALLSOLVE_H
#define SMALLSOLVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SS_MAX_N 4096

/* operations */
#define SS_OP_POTRF  0
#define SS_OP_TRSYL  1
#define SS_OP_TRLYAP 2

/* modes */
#define SS_MODE_FP64          0
#define SS_MODE_FP32_REFINED  1
#define SS_MODE_TF32_REFINED  2
#define SS_MODE_BF16_REFINED  3
#define SS_MODE_FP32_RAW      4
#define SS_MODE_TF32_RAW      5
#define SS_MODE_BF16_RAW      6
#define SS_NUM_MODES          7   /* modes 0..6 above; SS_MODE_DF is numbered after SS_MODE_AUTO */
#define SS_MODE_AUTO          7   /* per-size (mode, cfg) table, see ss_set_auto_table */
#define SS_MODE_DF            8   /* double-float block updates, FP64 diagonal blocks */

/* configuration selectors */
#define SS_CFG_DEFAULT (-1)
#define SS_CFG_TABLE   (-2)

/* return and info codes */
#define SS_ERR_CUDA       (-100)
#define SS_ERR_SCRATCH_LIMIT (-101)
#define SS_INFO_BAD_SIZE  (-1)
#define SS_INFO_NO_WORK   (-2)
#define SS_INFO_ALIASED   (-3)
#define SS_INFO_RANGE     (-4)
#define SS_INFO_TIMEOUT   (-5)

#define SS_ERR_IO          (-102)
#define SS_ERR_NO_SELECTOR (-103)

/* size bins of the configuration tables: bin(n) = ceil(log2(max(n, 1))) */
#define SS_NUM_BINS 13

#define SS_REFINE_MAXIT 10
#define SS_REFINE_TOL   1e-13

/*
 * Upper Cholesky X^T X = A (Fig. 2a).  Reads the upper triangle of A, writes
 * the upper triangle of X with a positive diagonal.
 */
int potrf_upper(int batch, int max_n, const int *d_n,
                const double *const *d_A, const int *d_lda,
                double *const *d_X, const int *d_ldx, int *d_info,
                int mode, int cfg, void *d_work, size_t work_bytes, void *stream);

/*
 * Triangular Sylvester L X + X U = C (Fig. 2c).  Reads the lower triangle of
 * L, the upper triangle of U and all of C; writes all of X.
 */
int trsyl_lu(int batch, int max_n, const int *d_n,
             const double *const *d_L, const int *d_ldl,
             const double *const *d_U, const int *d_ldu,
             const double *const *d_C, const int *d_ldc,
             double *const *d_X, const int *d_ldx, int *d_info,
             int mode, int cfg, void *d_work, size_t work_bytes, void *stream);

/*
 * Rectangular triangular Sylvester L X + X U = C with L (m x m) lower, U
 * (n x n) upper, C and X m x n.  The paper states the Sylvester problem for
 * n x n matrices (Fig. 2c); the equation and its recurrence hold unchanged for
 * m != n, which this entry point solves (a generalisation, not in the paper).
 * Per instance: m = d_m[b] rows, n = d_n[b] columns; d_ldl[b] >= max(1, m),
 * d_ldu[b] >= max(1, n), d_ldc[b] and d_ldx[b] >= max(1, m).  Reads the lower
 * triangle of L, the upper triangle of U and all of C; writes all of X (X may
 * alias C with the same leading dimension).  0 <= d_m[b] <= max_m and
 * 0 <= d_n[b] <= max_n, both bounds <= SS_MAX_N; an instance outside them gets
 * SS_INFO_BAD_SIZE and is left untouched; m = 0 or n = 0 is empty (info 0).
 * info = 1 when some |l_ii + u_jj| <= max(m, n) * DBL_EPSILON * max diagonal
 * magnitude of L and U, or is NaN.  Instances are scheduled longest-first by
 * max(m, n).  mode must be SS_MODE_FP64 or SS_MODE_DF (other modes return -15); cfg as for
 * trsyl_lu (the Sylvester configurations and tables).  Workspace: the size
 * ss_workspace_size(SS_OP_TRSYL, batch, max(max_m, max_n), mode, ...)
 * reports.
 */
int trsyl_rect(int batch, int max_m, int max_n, const int *d_m, const int *d_n,
               const double *const *d_L, const int *d_ldl,
               const double *const *d_U, const int *d_ldu,
               const double *const *d_C, const int *d_ldc,
               double *const *d_X, const int *d_ldx, int *d_info,
               int mode, int cfg, void *d_work, size_t work_bytes, void *stream);

/*
 * SPD solve A X = B through the upper Cholesky factor: R with R^T R = A
 * (Fig. 2a, computed as by potrf_upper), then R^T Y = B and R X = Y.  The
 * paper names the factorisation as a building block of linear-system solves;
 * this entry point is that use of it (not a problem the paper states).
 * Per instance: A is n x n (n = d_n[b], upper triangle read), R is written in
 * its upper triangle (d_R[b] may alias d_A[b] with the same leading
 * dimension; the strict lower triangle of R is left untouched), B and X are
 * n x k (k = d_k[b]; X may alias B with the same leading dimension).
 * d_ldr[b] >= max(1, n); d_ldb[b], d_ldx[b] >= max(1, n).  0 <= n <= max_n
 * <= SS_MAX_N and 0 <= k <= max_k.  info: 0 success; j > 0 the factor's
 * pivot j failed (X untouched); SS_INFO_BAD_SIZE for n or k out of range (X
 * untouched; for a bad k, R is computed).  mode must be SS_MODE_FP64 or
 * SS_MODE_DF (in DF the factor's and the triangular solves' block updates are
 * double-float, their diagonal blocks FP64; other modes return -15); cfg
 * selects the Cholesky configuration (as for potrf_upper in that mode).
 * Workspace: the size ss_workspace_size(SS_OP_POTRF, batch, max_n, mode, ...)
 * reports.  After the pre-passes, two launches: the factor, then the solves,
 * ordered on `stream`.
 */
int posv_upper(int batch, int max_n, int max_k, const int *d_n, const int *d_k,
               const double *const *d_A, const int *d_lda,
               double *const *d_R, const int *d_ldr,
               const double *const *d_B, const int *d_ldb,
               double *const *d_X, const int *d_ldx, int *d_info,
               int mode, int cfg, void *d_work, size_t work_bytes, void *stream);

/*
 * Triangular Lyapunov L X + X L^T = S (Fig. 2b).  Reads the lower triangles of
 * L and S; writes the lower triangle of the symmetric X.
 */
int trlyap_l(int batch, int max_n, const int *d_n,
             const double *const *d_L, const int *d_ldl,
             const double *const *d_S, const int *d_lds,
             double *const *d_X, const int *d_ldx, int *d_info,
             int mode, int cfg, void *d_work, size_t work_bytes, void *stream);

/*
 * Workspace, in bytes, that a call of `op` with this batch, max_n and mode
 * needs (the bound assumes every instance has order max_n; for SS_MODE_AUTO
 * it covers whichever modes the table may choose).  Returns 0 and
 * writes *bytes, or a negative argument error.
 */
int ss_workspace_size(int op, int batch, int max_n, int mode, size_t *bytes);

/*
 * Kernel configurations.  ss_config_count returns how many explicit
 * configurations `op` has in `mode` (or a negative error);
 * ss_config_describe writes the block size, threads per CTA and algorithm
 * variant of configuration `cfg` (any pointer may be NULL).  In the TF32 and
 * BF16 refined modes, variant bit 2 marks the tensor-memory configurations:
 * the low-precision solve keeps its trailing matrix (Cholesky, n <= 256) or
 * right-hand side (Sylvester / Lyapunov, n <= 128) in tensor memory and
 * applies the trailing updates with tcgen05 MMAs; larger instances of the
 * same call take the blocked / warp-block path.
 */
int ss_config_count(int op, int mode);
int ss_config_describe(int op, int mode, int cfg, int *block, int *threads, int *variant);

/*
 * Per-size configuration table used by cfg = SS_CFG_TABLE.  cfg_by_n[k] is the
 * configuration for instances of order n with bin(n) = k, where bin(n) =
 * ceil(log2(max(n, 1))) (so bins 0..12 cover n up to 4096); -1 means the
 * built-in default.  The table is host-side library state, copied; setting
 * nbins = 0 clears it.  Calls are not thread-safe with concurrent solves.
 */
int ss_set_config_table(int op, int mode, int nbins, const int *cfg_by_bin);

/*
 * trsyl_lu without a workspace argument, for callers that cannot allocate
 * device memory (the paper has no counterpart; this is a library interface
 * choice).  Same arguments, layout and info codes as trsyl_lu in
 * SS_MODE_FP64 with SS_CFG_DEFAULT, minus d_work/work_bytes: the scratch is a
 * fixed 1 MiB area in the library's own device memory, held on every device
 * that loads the library until the process exits.  That is enough for any
 * batch up to 261952 instances (any max_n); a larger batch returns
 * SS_ERR_SCRATCH_LIMIT before anything is launched.  The first call on each
 * device looks the area's address up (cudaGetSymbolAddress) with that device
 * current, so make it before any stream capture.  All calls share the area:
 * calls that overlap on the GPU race and must be ordered.  Allocates nothing.
 */
int trsyl_lu_noalloc(int batch, int max_n, const int *d_n,
                     const double *const *d_L, const int *d_ldl,
                     const double *const *d_U, const int *d_ldu,
                     const double *const *d_C, const int *d_ldc,
                     double *const *d_X, const int *d_ldx, int *d_info, void *stream);

/*
 * Per-size (mode, cfg) table used by mode = SS_MODE_AUTO: bin k (bin(n) as for
 * ss_set_config_table) runs in mode_by_bin[k] (SS_MODE_FP64 or one of the
 * *_REFINED modes; -1 = unset) with configuration cfg_by_bin[k] (-1 = that
 * mode's default).  nbins = 0 clears the table.  Host-side state, copied.
 */
int ss_set_auto_table(int op, int nbins, const int *mode_by_bin, const int *cfg_by_bin);

/*
 * The learned selector's cost model (the paper's "Limitations and future
 * work" paragraph: replace the autotuning loops with a model-based approach).
 * A fixed MLP  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3
 * maps SS_MLP_IN features (op one-hot [3], log2 n, log2 batch, mode one-hot
 * [FP64, FP32, TF32, BF16 refined, DF]) to SS_MLP_OUT predicted log2 run times,
 * one per kernel configuration id.  Parameters: one device float array of
 * SS_MLP_PARAMS values laid out W1 (H x IN, row-major), b1, W2 (H x H), b2,
 * W3 (OUT x H), b3.  All arrays are device pointers, row-major per row.
 *
 * ss_mlp_forward: y[nrows x OUT] = MLP(x[nrows x IN]).
 * ss_mlp_grad: loss = sum mask (y - t)^2 / mask_total and its gradient with
 *   respect to every parameter (written to d_grad[SS_MLP_PARAMS], loss to
 *   *d_loss); mask_total must be the sum of the mask (> 0).  Needs
 *   ss_mlp_workspace_size(nrows) bytes of workspace.  Deterministic.
 * ss_mlp_adam: one Adam step (bias-corrected, step >= 1) updating d_params
 *   and the moment arrays d_m, d_v (each SS_MLP_PARAMS floats, zero at start).
 * Return 0, -k for an invalid argument k, or SS_ERR_CUDA.
 */
#define SS_MLP_IN 10
#define SS_MLP_HIDDEN 64
#define SS_MLP_OUT 8
#define SS_MLP_PARAMS (SS_MLP_HIDDEN * SS_MLP_IN + SS_MLP_HIDDEN + SS_MLP_HIDDEN * SS_MLP_HIDDEN + \
                       SS_MLP_HIDDEN + SS_MLP_OUT * SS_MLP_HIDDEN + SS_MLP_OUT)
int ss_mlp_workspace_size(int nrows, size_t *bytes);
int ss_mlp_forward(const float *d_params, int nrows, const float *d_x, float *d_y, void *stream);
int ss_mlp_grad(const float *d_params, int nrows, const float *d_x, const float *d_t,
                const float *d_mask, float mask_total, float *d_grad, float *d_loss,
                void *d_work, size_t work_bytes, void *stream);
int ss_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int step, float lr,
                float beta1, float beta2, float eps, void *stream);

/*
 * The autotuner (the paper's search loop over algorithm variants and
 * implementation parameters, "Generator structure" paragraph) on one batch:
 * every configuration of `mode` (0 <= cfg < ss_config_count(op, mode)) is
 * run once to warm up and then `reps` times, each call timed with CUDA
 * events on `stream`; h_ms[cfg] gets the median milliseconds, h_bad[cfg]
 * (may be NULL) the number of instances whose info was nonzero, and
 * *best_cfg the fastest configuration whose solves all succeeded (-1: none).
 * The operands are those of the entry point of `op`: potrf_upper takes d_A;
 * trsyl_lu takes L = d_A, U = d_B, C = d_C; trlyap_l takes L = d_A,
 * S = d_C (d_B unused); X, info and the workspace as there (sized for
 * `mode`).  mode is any mode but SS_MODE_AUTO.  This is a tuning call, not
 * part of the solve path: it synchronises `stream` and cannot be captured
 * in a CUDA graph.  h_ms and h_bad hold ss_config_count(op, mode) entries.
 * Returns 0, -k for an invalid argument k, or the error of the first
 * failing solve call.
 */
int ss_autotune(int op, int mode, int batch, int max_n, const int *d_n,
                const double *const *d_A, const int *d_lda,
                const double *const *d_B, const int *d_ldb,
                const double *const *d_C, const int *d_ldc,
                double *const *d_X, const int *d_ldx, int *d_info,
                void *d_work, size_t work_bytes, int reps,
                float *h_ms, int *h_bad, int *best_cfg, void *stream);

/*
 * The learned selector (the paper's "Limitations and future work"
 * paragraph: model-based selection instead of autotuning): the MLP above,
 * evaluated for every (precision mode, configuration) of a call, predicts
 * which one is fastest.  Library state, one model per process, guarded by a
 * lock.
 *
 * Model: the SS_MLP_PARAMS parameters; cfg_count[op * 5 + m] (may be NULL:
 * every configuration), the configurations of (op, selector mode m) that had
 * training targets; batch_max[(op * SS_NUM_BINS + k) * 5 + m] (may be NULL:
 * no limit), the largest batch trained for size bin k, beyond which a
 * prediction is taken at that batch and scaled linearly with the count.
 * Selector modes m = 0..4 are SS_MODE_FP64, SS_MODE_FP32_REFINED,
 * SS_MODE_TF32_REFINED, SS_MODE_BF16_REFINED and SS_MODE_DF (the modes that
 * meet the FP64 accuracy gate); the features of a (op, n, batch, m) query are
 * op one-hot [3], log2(n) / 9, log2(batch) / 14, m one-hot [5], with n the
 * geometric centre of the size bin.
 *
 * ss_selector_set / ss_selector_get: copy a model in or out (host arrays;
 * get: -1 if none is set).  ss_selector_clear: forget it.
 * ss_selector_save / ss_selector_load: the model as a little-endian binary
 * file ("SSMLP1" header, dimensions, parameters, cfg_count, batch_max);
 * SS_ERR_IO on a missing, short or mismatched file.
 * ss_selector_train: Adam on the masked mean squared error of log2 ms
 * targets (ss_mlp_grad / ss_mlp_adam, beta1 0.9, beta2 0.999, eps 1e-8,
 * `steps` steps at rate lr) from h_init (NULL: the current model), rows of
 * h_x [rows x SS_MLP_IN], h_t and h_m [rows x SS_MLP_OUT]; h_loss (may be
 * NULL) gets the loss before each step.  The trained parameters, and
 * cfg_count and batch_max read off the rows' features and mask, become the
 * model.  Allocates and frees its device buffers; synchronises `stream`.
 *
 * A call with count_by_bin[k] instances in size bin k (k < nbins):
 * ss_selector_queries writes the feature rows to evaluate (at most
 * SS_SELECTOR_MAX_ROWS) and their number; ss_selector_decide turns the
 * network's outputs for them, h_y [nrows x SS_MLP_OUT] log2 ms, into a
 * (mode, cfg) per bin: SS_SELECTOR_PER_BIN the fastest per bin,
 * SS_SELECTOR_CALL the single pair with the smallest predicted total over the
 * call, written to every bin (one launch group); bins without a choice get
 * -1; *pred_ms (may be NULL) the predicted total.  ss_selector_predict does
 * both around the CUDA forward kernel on `stream` (synchronised; the model's
 * device copy and row buffers are allocated on a device's first prediction
 * and kept).  ss_selector_install predicts and passes the result to
 * ss_set_auto_table.  All return 0, -k for an invalid argument k,
 * SS_ERR_NO_SELECTOR without a model, or SS_ERR_CUDA.
 */
#define SS_SELECTOR_PER_BIN 0
#define SS_SELECTOR_CALL 1
#define SS_SELECTOR_MAX_ROWS (SS_NUM_BINS * 5)
int ss_selector_set(const float *h_params, const int *cfg_count, const int *batch_max);
int ss_selector_get(float *h_params, int *cfg_count, int *batch_max);
int ss_selector_clear(void);
int ss_selector_save(const char *path);
int ss_selector_load(const char *path);
int ss_selector_train(const float *h_x, const float *h_t, const float *h_m, int rows, const float *h_init,
                      int steps, float lr, float *h_loss, void *stream);
int ss_selector_queries(int op, int nbins, const int *count_by_bin, float *h_x, int *nrows);
int ss_selector_decide(int op, int nbins, const int *count_by_bin, int policy, const float *h_y,
                       int *mode_by_bin, int *cfg_by_bin, double *pred_ms);
int ss_selector_predict(int op, int nbins, const int *count_by_bin, int policy,
                        int *mode_by_bin, int *cfg_by_bin, double *pred_ms, void *stream);
int ss_selector_install(int op, int nbins, const int *count_by_bin, int policy, void *stream);

/*
 * Tensor-core self-test (no counterpart in the paper): one 128 x n tile on
 * the fifth-generation tensor cores through the operand layout, descriptors,
 * tensor-memory accumulator and completion path that the refined modes'
 * trailing updates use, so that the encodings can be checked against a host
 * product.  D = op(A) B^T, or D = C + op(A) B^T with flags bit 0; op(A) = -A
 * with flags bit 1 (the instruction's negate-A bit).  Device arrays, FP32,
 * row-major: A 128 x k, B n x k, C and D 128 x n.  kind 0: the operands are
 * rounded to TF32 (k a multiple of 8), kind 1: to BF16 (k a multiple of 16);
 * 16 <= n <= 256 with n % 16 == 0, k <= 64.  One CTA on `stream`; *d_status
 * = 0 when the tile completed, 1 if the bounded wait for it ran out (D is
 * then unwritten).  Returns 0, -k for an invalid argument k, or SS_ERR_CUDA.
 */
int ss_umma_selftest(int kind, int n, int k, const float *d_a, const float *d_b, const float *d_c, float *d_d,
                     int flags, int *d_status, void *stream);

/* Library version. */
int ss_version(void);

/*
 * Instrumentation for benchmarks (no counterpart in the paper).
 * ss_launch_count: number of kernels this library has launched in this
 * process so far (all entry points, all devices).
 * ss_profile_enable(1): from now on, every solve call also records a CUDA
 * event pair on its stream around its solve kernels (after the binning
 * pre-pass, after the last solve launch).  ss_profile_read waits for the
 * recorded pairs, returns their total elapsed milliseconds and count, and
 * forgets them.  ss_profile_enable(0) stops recording.  Events are created on
 * first use and reused; this is host-side state, not thread-safe with
 * concurrent calls.  Returns 0 or a negative error.
 */
long long ss_launch_count(void);
int ss_profile_enable(int on);
int ss_profile_read(double *total_ms, int *calls);

#ifdef __cplusplus
}
#endif

#endif /* SMALLSOLVE_H */
