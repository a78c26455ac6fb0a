/*
 * rs.h -- C ABI of the GB300 (sm_103a) library for the tier-2 / tier-3 analysis of an
 * optimization-recommendation tool (Taheri, Qasem, Burtscher: "A Tool for Automatically
 * Suggesting Source-Code Optimizations for Complex GPU Kernels").
 *
 * The tool's tiers talk through a simple interface so that any tier can be replaced
 * (Sec. 2).  This header is that interface for tiers 2 and 3: profiled feature vectors in,
 * per-optimization predicted speedups out, sorted, thresholded and truncated.
 *
 * Conventions for every entry point
 *   - Pointers named in a struct or argument list are DEVICE pointers unless the comment
 *     says "host".  All of them are owned by the caller; the library never frees them.
 *   - Calls are asynchronous on the stream given to rs_create (or rs_set_stream).  A
 *     return of RS_OK means the work was enqueued; results are valid after the stream is
 *     synchronised.
 *   - A call that returns anything but RS_OK enqueued nothing (argument errors) or hit a
 *     CUDA error; rs_last_error gives a one-line reason.  Problems of a single fit
 *     (no training pair, a non-positive pivot, a non-finite value) are not errors: they go
 *     to the per-fit status array and never abort a batch.
 *   - Data layout: a batch holds P programs; program p owns the versions (rows)
 *     row_offsets[p] .. row_offsets[p+1]-1 (at most 64, one per 6-bit optimization mask,
 *     Sec. 3.3) and a row-major [V_p][F_p] counter block starting at element x_offsets[p]
 *     of X.  Per-feature statistics of program p sit at feat_offsets[p] + f.
 *   - A split trains on the version slots whose bit is set in its 64-bit train mask (bit r
 *     = the program's r-th row) and tests on the other slots (Sec. 5).  Splits of
 *     program p are split_offsets[p] .. split_offsets[p+1]-1.
 */
#ifndef RS_H_
#define RS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RS_OK = 0,
    RS_EINVAL = 1,        /* bad argument (null pointer, size out of range, bad enum)   */
    RS_ENOMEM = 2,        /* a caller-provided workspace is too small                   */
    RS_ECUDA = 3,         /* a CUDA runtime call failed                                 */
    RS_ETIMEOUT = 4,      /* a bounded device-side wait gave up                         */
    RS_EUNSUPPORTED = 5,  /* the device is not sm_103 / feature not built               */
    RS_EDATA = 6          /* the device found inconsistent data (see rs_last_error)      */
} rs_status;

enum { RS_FIT_OK = 0, RS_FIT_EMPTY = 1, RS_FIT_NOTPD = 2, RS_FIT_NONFINITE = 3 };
enum { RS_F32 = 0, RS_F64 = 1 };
/* Gram precision: plain FP64 FMAs, or the BF16 hi/lo split on the tensor cores (three
 * BF16 products per term, FP32 accumulation in tensor memory).  RS_GRAM_DIST2 makes the
 * block of squared Euclidean distances instead, for the instance-based learner.         */
enum { RS_GRAM_F64 = 0, RS_GRAM_BF16X3 = 1, RS_GRAM_DIST2 = 2 };
/* Fit forms: the batched form (fits binned by size, one thread per small fit), or the
 * plain form (one warp per fit, lanes = matrix rows).  Both give the same results.     */
enum { RS_FORM_BATCHED = 0, RS_FORM_PLAIN = 1 };
/* Flags for rs_predict_rank. */
enum {
    RS_RANK_ALL = 1,      /* rank all six optimizations, not only those not yet applied */
    RS_REFINE_X = 2,      /* one step of iterative refinement with residual and
                             predictions taken through Z (for an inexact Gram)        */
    RS_MODEL_IBK = 4,     /* the instance-based learner (IBK, k nearest neighbours)
                             instead of ridge regression; K is the distance block    */
    RS_MODEL_M5P = 8,     /* the M5P model tree instead of ridge regression (rs_transfer) */
    RS_PACK_PRED = 16,    /* rec_pred packed: the reported lists back to back (rs_predict_rank) */
    RS_LOO_CLOSED = 32    /* leave-one-version-out splits: every fit from one inverse of its
                             program's full system (rs_predict_rank, rs_cv_step)      */
};
#define RS_IBK_NEIGHBORS 10  /* k of the instance-based learner (Sec. 3.4: k = 10)        */

#define RS_NOPT 6
#define RS_MAXV 64          /* versions per program (6-bit masks)                       */
#define RS_MAXPAIRS 32      /* pairs per optimization per program                        */
#define RS_COEF_STRIDE 33   /* doubles per fit in the coefficient array: b, alpha[32]   */
#define RS_GRAM_LD 64       /* leading dimension of each program's Gram block           */
#define RS_MAXRUNS 4        /* runs in one training group of rs_transfer                 */
#define RS_NCOUNTERS 16

/* Accuracy counters (uint64, accumulated, never reset by the library):
 *  0 test rows ranked        1 predictions made          2 predictions with a known actual
 *  3 sign hits (pred > 0 and actual > 0 agree: the accuracy of Table 3)
 *  4 recommendations emitted 5 ... with a known actual   6 ... whose actual speedup > 1
 *  7 rows with >= 1 scored prediction  8 ... whose top prediction is the best actual
 *  9..12 fits by status OK / EMPTY / NOTPD / NONFINITE (rs_predict_rank, rs_transfer)
 * 13 candidates skipped because their fit was not OK     14, 15 reserved (0)          */

typedef struct rs_ctx rs_ctx;

typedef struct {
    int32_t n_programs;          /* host: P >= 1                                          */
    int32_t dtype;               /* host: RS_F32 or RS_F64, element type of X             */
    int64_t n_rows;              /* host: total versions = row_offsets[P]                 */
    int32_t max_versions;        /* host: upper bound on V_p, 1..64                       */
    int32_t max_feat;            /* host: upper bound on F_p, 1..4096                     */
    int64_t x_elems;             /* host: elements of X (and of Z)                        */
    int64_t feat_total;          /* host: sum of F_p = feat_offsets[P]                    */
    const int64_t* row_offsets;  /* [P+1]                                                 */
    const int32_t* feat_width;   /* [P]                                                   */
    const int64_t* x_offsets;    /* [P]                                                   */
    const int64_t* feat_offsets; /* [P+1]                                                 */
    const void* X;               /* raw counters (dtype), or standardized Z (double)      */
    const uint8_t* masks;        /* [n_rows] 6-bit optimization mask of each version      */
    const double* log_time;      /* [n_rows] log run time of each version                 */
    const double* cycles;        /* [n_rows] cycle counts, or NULL (no normalisation)     */
} rs_batch;

typedef struct {
    int64_t n_splits;            /* host: S = split_offsets[P]                            */
    int64_t n_test_rows;         /* host: rec_offsets[S] if known, else 0 (then the bound
                                    S * max_versions sizes the prediction buffer)         */
    int32_t max_train;           /* host: upper bound on popcount(train mask), 0..64      */
    int32_t reserved;
    const int64_t* split_offsets;/* [P+1]                                                 */
    const uint64_t* train_masks; /* [S]                                                   */
} rs_splits;

/* ---- context ------------------------------------------------------------------------
 * rs_create: binds a context to CUDA device `device` and the stream `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  Allocates 4 KiB of device memory for
 * the context's status word and queue heads and 32 KiB for the row-planning scan.
 * Fails with RS_EUNSUPPORTED if the device is not compute capability 10.3.
 * rs_destroy frees them.                                                              */
rs_status rs_create(rs_ctx** out, int device, void* cuda_stream);
rs_status rs_destroy(rs_ctx* ctx);
rs_status rs_set_stream(rs_ctx* ctx, void* cuda_stream);
/* Last error of this context as a NUL-terminated string ("" if none); owned by ctx.   */
const char* rs_last_error(const rs_ctx* ctx);
/* Reads (and clears) the device status word after a stream sync: RS_OK, RS_EDATA when a
 * kernel met a program with more than 64 versions or more pairs than the hint allowed,
 * RS_ETIMEOUT when a bounded wait gave up.  Synchronises the context's stream.        */
rs_status rs_check_device_status(rs_ctx* ctx);
/* Stage timing (a tracing aid, not part of the method).  rs_profile_enable(ctx, 1) makes
 * the batched fit/predict path record CUDA events on the context's stream around each of
 * its six internal launches (pair tables, fit planning, bucketing, small solves, large
 * solves, rank); rs_profile_read waits for the last event and writes the six stage
 * durations in milliseconds of the most recent batched call into ms (at most max_stages;
 * *n_stages = count).  RS_EINVAL if profiling is off.                                */
rs_status rs_profile_enable(rs_ctx* ctx, int on);
rs_status rs_profile_read(rs_ctx* ctx, float* ms, int max_stages, int* n_stages);

/* ---- A1: feature vectors (Sec. 2) -----------------------------------------------------
 * Z[r][f] = (log(max(X[r][f] / cycles[r], 1e-30)) - mu_f) / sigma_f with mu_f, sigma_f the
 * population mean and standard deviation of the log values over the program's versions
 * (sigma_f < 1e-12 gives Z = 0).  The division by the cycle count is the paper's
 * normalisation (Sec. 2); the log and z-score are this library's reading.
 * Z: double, same layout as X (x_elems).  mu, sigma: double [feat_total], may be NULL.
 * All arithmetic is FP64 whatever the input type.                                     */
rs_status rs_standardize(rs_ctx* ctx, const rs_batch* batch, double* Z, double* mu,
                         double* sigma);

/* ---- A3: per-program Gram of the standardized feature vectors -------------------------
 * K_p[a][b] = sum_f Z[a][f] * Z[b][f] for a, b < V_p, written to
 * K[p * 64 * 64 + a * 64 + b] (double; entries outside V_p x V_p are left untouched).
 * std: a batch whose X is Z (double).  precision: RS_GRAM_F64 (FP64 FMAs, no workspace) or
 * RS_GRAM_BF16X3 (tcgen05 tensor cores: z = hi + lo with hi = bf16(z), lo = bf16(z - hi),
 * K ~ hi hi^T + hi lo^T + lo hi^T accumulated in FP32 -- relative error about 2^-16 per
 * entry; symmetric; needs rs_gram_workspace_bytes(std, precision) bytes of workspace,
 * 256-byte aligned, and at most 65535 programs per call).  Every ridge fit of a split reads
 * its kernel entries from this block (the dual form of the regression).
 * RS_GRAM_DIST2 (no workspace): K_p[a][b] = sum_f (Z[a][f] - Z[b][f])^2, the squared
 * Euclidean distances of the instance-based learner (Sec. 3.4), each summed in ascending f
 * with one rounding per subtraction, product and addition (no fused multiply-add), so the
 * entries are those of the plain definition.                                          */
size_t rs_gram_workspace_bytes(const rs_batch* std, int precision);
rs_status rs_gram(rs_ctx* ctx, const rs_batch* std, int precision, double* K, void* workspace,
                  size_t workspace_bytes);

/* ---- A2: test-row planning ------------------------------------------------------------
 * rec_offsets[i] = number of test rows (version slots outside the train mask) of all
 * splits before split i; rec_offsets[S] = total.  int64 [S+1].  Rows of a split are in
 * ascending slot order.  Every rs_predict_rank output is indexed by these rows.       */
rs_status rs_rec_offsets(rs_ctx* ctx, const rs_batch* batch, const rs_splits* splits,
                         int64_t* rec_offsets);

/* ---- A2 + A4: batched ridge fits (Sec. 2 tier-2 training, Sec. 3.4 regression) ---------
 * For every split and optimization j: the training pairs are the before/after version
 * pairs (v, v|j) with both versions in the train mask (Sec. 3.3); each pair contributes
 * the feature vector of v labelled with log t(v) - log t(v|j), the log speedup of adding
 * j (Sec. 5).  Fits minimise sum (y - b - z.beta)^2 + lambda |beta|^2 with an unpenalised
 * intercept, solved in dual form from the Gram block K with an FP64 Cholesky:
 * beta = sum_a alpha_a z_a.
 * coef (nullable): double [S][6][33] = b, then alpha for the training pairs in ascending
 * order of their before-version slot (zeros after n); b is NaN when the fit is not OK.
 * fit_status (nullable): uint8 [S][6] RS_FIT_*.  lambda >= 0 (at lambda = 0 the dual
 * system is the minimum-norm interpolant when n <= F).
 * form: RS_FORM_BATCHED (fits of the whole batch sorted by size, one thread per fit up to
 * 10 pairs, lanes sharing the larger fits) or RS_FORM_PLAIN (one warp per fit, per chunk);
 * with the batched form, form | RS_REFINE_X takes one step of iterative refinement of every
 * fit through the standardized features of `std` (for a K from RS_GRAM_BF16X3), as the
 * flag does in rs_predict_rank; form | RS_LOO_CLOSED (batched, not with RS_REFINE_X) takes
 * the fits of leave-one-version-out splits in closed form, as in rs_predict_rank.
 * workspace: caller-owned device scratch of at least rs_fit_workspace_bytes(std, splits)
 * bytes, 256-byte aligned, required by the batched form (may be NULL for the plain form);
 * its contents are undefined after the call.  RS_ENOMEM if it is too small.  A fit with
 * more pairs than splits->max_train / 2 (a wrong hint) is treated as empty and the device
 * status reports RS_EDATA.                                                            */
size_t rs_fit_workspace_bytes(const rs_batch* std, const rs_splits* splits);
rs_status rs_fit_batched(rs_ctx* ctx, const rs_batch* std, const double* K,
                         const rs_splits* splits, double lambda, int form, void* workspace,
                         size_t workspace_bytes, double* coef, uint8_t* fit_status);

/* ---- A4 + A5 + A6: fit, predict, rank, threshold, score (Sec. 2 tier 3, Sec. 5, 6) -----
 * For every test row t of every split: one predicted log speedup per candidate
 * optimization (those not in t's mask; all six with RS_RANK_ALL), b + sum_a alpha_a
 * K[t][v_a] from the split's fit; candidates sorted by prediction (ties: lower index
 * first), kept if >= log(tau), at most k (1..6) reported.  The fits are computed in the
 * same call (as rs_fit_batched with the same form and workspace rules) unless coef, from
 * rs_fit_batched with the same inputs, is given; then no workspace is needed.
 * rec_offsets: from rs_rec_offsets.  Outputs per row (R = rec_offsets[S]):
 *   rec_code  uint32 [R]: bits 0-3 = count c, bits 4+4i..7+4i = i-th optimization (0xF unused)
 *   rec_pred  double [R][k]: predicted log speedups of the reported list (NaN unused), nullable
 *             with RS_PACK_PRED (batched form, fits in the call): packed instead, row r's c_r
 *             reported predictions at rec_pred[P_r .. P_r + c_r - 1], P_r = sum of c over the
 *             rows before r (c from rec_code; the total is counter 4 when counters are
 *             given), no NaN padding -- about 1.2 values per row instead of k
 *   pred_all  double [R][6]: every prediction (NaN where none), nullable
 *   counters  uint64 [16]: accuracy counters (listed above), added to; nullable
 * flags: RS_RANK_ALL; RS_REFINE_X (batched form, coef == NULL): every fit gets one step of
 * iterative refinement of its bordered system with the residual computed from Z in FP64
 * (r_a = y_a - b - lambda alpha_a - z_a . beta, beta = sum_a alpha_a z_a), solved with the
 * same factor, and predictions are taken through Z (b + z_t . beta) -- for Gram blocks made
 * with RS_GRAM_BF16X3.  RS_MODEL_IBK (batched form, coef == NULL, not with RS_REFINE_X; K
 * from rs_gram with RS_GRAM_DIST2): the instance-based learner of Sec. 3.4 replaces the
 * regression -- a fit is OK when it has a training pair; the prediction for test row t is
 * the mean label of the RS_IBK_NEIGHBORS training pairs whose before versions are nearest
 * to t (distance K[t][v_a]; equal distances take the lower pair first; all pairs when there
 * are fewer), summed in ascending pair order.  lambda is ignored.  RS_LOO_CLOSED (batched
 * form, coef == NULL, not with RS_REFINE_X or RS_MODEL_IBK): for splits that each hold out
 * one version (the leave-one-version-out protocol of Sec. 5), optimization j's training
 * pairs are the program's pairs for j minus at most the one that contains the held-out
 * version, so every fit is the program's full system M = K_PP + lambda I without one row and
 * column.  With M^-1, w_y = M^-1 y and w_1 = M^-1 1 formed once per (program, j), the
 * reduced system's M_r^-1 y = (w_y - u w_y[i] / u_i) without entry i (u = column i of M^-1)
 * and likewise for 1, so b and alpha cost O(n) per fit instead of a factorization.  The same
 * fits to rounding (the inverse adds an error of order cond(M) times the unit roundoff) and the
 * same statuses.  A fit whose split leaves out more than one of its program's pairs for j
 * (a split that holds out two or more versions, in general) has no such form: RS_EDATA
 * (detail: the program), and the fit is reported failed (RS_FIT_NOTPD).  tau > 0.     */
rs_status rs_predict_rank(rs_ctx* ctx, const rs_batch* std, const double* K,
                          const rs_splits* splits, double lambda, const double* coef,
                          int k, double tau, int flags, int form, void* workspace,
                          size_t workspace_bytes, const int64_t* rec_offsets,
                          uint32_t* rec_code, double* rec_pred, double* pred_all,
                          uint64_t* counters);

/* ---- the whole step in one call ---------------------------------------------------------
 * rs_cv_step runs A1..A6 on raw counters: standardize into workspace, Gram (precision as
 * given), plan rows into rec_offsets, then the batched fit/predict/rank.  workspace:
 * device memory of at least rs_cv_workspace_bytes(batch, splits) bytes, 256-byte
 * aligned, owned by the caller and used as scratch (Z, the Gram blocks and the fit
 * workspace).  Outputs as in rs_predict_rank, equal bit for bit to those of the individual
 * calls.  With RS_MODEL_IBK the block is the distance block (precision RS_GRAM_F64 or
 * RS_GRAM_DIST2).  Ordering: the row planning and the fit plan (they read only masks, times
 * and splits) run on the context's internal second stream beside the standardization and
 * the Gram, forked from and joined back into the context's stream with events, so the call
 * is still ordered on the context's stream as a whole; with RS_GRAM_BF16X3 (whose scratch is
 * the fit workspace) every stage runs on the context's stream in order.  One context must
 * not run two calls at once from different host threads.                                */
size_t rs_cv_workspace_bytes(const rs_batch* batch, const rs_splits* splits);
rs_status rs_cv_step(rs_ctx* ctx, const rs_batch* batch, const rs_splits* splits,
                     double lambda, int k, double tau, int flags, int precision,
                     void* workspace, size_t workspace_bytes, int64_t* rec_offsets,
                     uint32_t* rec_code, double* rec_pred, double* pred_all,
                     uint64_t* counters);

/* ---- Table 2: transfer to another run, input or program (Sec. 5) -------------------------
 * Q transfer problems.  Problem q trains on a group of runs of `train` -- runs
 * group_offsets[q] .. group_offsets[q+1]-1, each laid out like one program of a batch (at most
 * 64 versions with distinct masks), 1..max_runs of them -- and tests on program q of `test`
 * (Q = test->n_programs).  groups == NULL: one run per problem, run q for problem q (then
 * train->n_programs == Q).  The runs of a group and its test program have one feature width.
 * Both sets hold raw counters (dtype, cycles as in rs_standardize).  Per problem: the vectors
 * of all the group's runs are standardized together (mu, sigma over all of them, as
 * rs_standardize) and the test program with those statistics; per optimization j the model
 * is trained from every before/after pair (v, v|j) of every run of the group (a pair never
 * spans two runs), labelled with its run's log speedup -- ridge (lambda, FP64, the bordered
 * dual system of rs_fit_batched on up to 32 * max_runs pairs) or, with RS_MODEL_IBK, the
 * instance-based learner (as rs_predict_rank; pairs in run order, then ascending before
 * slot) -- and predicts for every version t of the test program each candidate j that is
 * outside t's mask (all six with RS_RANK_ALL) and inside opt_mask (bits of the optimizations
 * that may be recommended: 0x3F for all, fewer for transfer between programs that share only
 * some optimizations).  Ranking, threshold, top-k and scoring as in rs_predict_rank, the
 * actual speedups taken from the test program's own times.  Rows: the test set's versions in
 * order (R = test->n_rows).  Outputs (device memory): rec_code [R] (required), rec_pred
 * [R][k], pred_all [R][6], counters [16] (9..12 count the Q * 6 fits) and fit_status [Q][6]
 * (nullable).  A problem whose group or test program breaks these rules is skipped (its rows
 * are not written) and reported as RS_EDATA in the device status.  workspace: device memory
 * of at least rs_transfer_workspace_bytes(train, test, groups) bytes, 256-byte aligned,
 * scratch.  flags: RS_RANK_ALL, and RS_MODEL_IBK or RS_MODEL_M5P.  tau > 0, k in 1..6.
 * RS_MODEL_M5P (Sec. 3.4's model tree, after the published M5' description): per fit, a tree
 * grown by the standard deviation reduction (nodes of fewer than 4 instances, or whose label
 * deviation is at most 5 % of the root's, are leaves; thresholds halfway between consecutive
 * distinct values, at least 2 instances a side, ties to the lower attribute), a least-squares
 * model at every node on the attributes tested below it (at most 64), simplified by greedy
 * elimination on the estimated error mean|residual| (m + v) / (m - v), bottom-up pruning,
 * and smoothing on the way up, p = (n p + 15 q) / (n + 15); at most 256 features (else
 * RS_EUNSUPPORTED).  Its workspace (rs_transfer_workspace_bytes with the same flags) holds
 * the trees.                                                                             */
typedef struct {
    int64_t n_groups;             /* host: Q, equal to test->n_programs                      */
    int32_t max_runs;             /* host: upper bound on runs per group, 1..RS_MAXRUNS      */
    int32_t reserved;
    const int64_t* group_offsets; /* [Q+1] device: group_offsets[0] = 0, non-decreasing      */
} rs_groups;
size_t rs_transfer_workspace_bytes(const rs_batch* train, const rs_batch* test, const rs_groups* groups,
                                   int flags);
rs_status rs_transfer(rs_ctx* ctx, const rs_batch* train, const rs_batch* test, const rs_groups* groups,
                      double lambda, int k, double tau, int flags, int opt_mask, void* workspace,
                      size_t workspace_bytes, uint8_t* fit_status, uint32_t* rec_code, double* rec_pred,
                      double* pred_all, uint64_t* counters);

/* ---- A3 + A4, primal form: pooled ridge fits over many programs ----------------------------
 * One ridge model per optimization j (Sec. 3.4 regression family, the same loss as the batched
 * fits: minimise sum (y - b - z.beta)^2 + lambda |beta|^2, intercept unpenalised) trained on
 * the before/after pairs (v, v|j) of every program p of `std` with use_program[p] != 0
 * (device uint8 [P]; NULL = all programs), pairs formed within each program (Sec. 3.3),
 * labelled with its log speedup (Sec. 5): the model of a tool that has seen many codes.
 * With the pairs far outnumbering the F features the primal normal equations are solved:
 * G_j = sum_a c_a c_a^T + lambda I with c_a = z_a - zbar_j the centred feature vectors (the
 * Gram X^T W X, W selecting j's pairs), formed as ONE batched tcgen05 GEMM over the six j from a
 * BF16 hi/lo split of the centred rows (K = 3 x pairs, FP32 accumulation, TMA-fed), then an FP64
 * Cholesky; with RS_REFINE_X in flags one refinement step whose residual is taken exactly in
 * FP64 through the rows (recovering FP64 accuracy while kappa(G) * 2^-16 << 1).
 * std: standardized features (X = Z, double), one width F = max_feat (<= 512) for every
 * training program (a program of another width, or of more than 64 versions, is skipped
 * and reported as RS_EDATA); at most 65,535 programs and 65,536 pairs per optimization.
 * coef: double [6][F + 1] (device) = b_j, then beta_j; fit_status: uint8 [6] (device);
 * a fit without pairs is RS_FIT_EMPTY, a non-positive pivot RS_FIT_NOTPD (b = NaN).
 * workspace: rs_pooled_workspace_bytes(std) bytes, 256-byte aligned (RS_ENOMEM if smaller).
 * lambda > 0.  Asynchronous on the context's stream.
 * rs_predict_pooled: for every version t of `std` (rows in batch order) the predictions
 * b_j + z_t.beta_j of its candidate optimizations (not in t's mask; all six with
 * RS_RANK_ALL) whose fit is OK, ranked, thresholded at log(tau), top k and scored against
 * the version's own program (actual speedups from its times) exactly as rs_predict_rank
 * does: rec_code [n_rows], rec_pred [n_rows][k] (nullable), pred_all [n_rows][6]
 * (nullable), counters (nullable, added to).                                              */
size_t rs_pooled_workspace_bytes(const rs_batch* std);
rs_status rs_fit_pooled(rs_ctx* ctx, const rs_batch* std, const uint8_t* use_program, double lambda,
                        int flags, void* workspace, size_t workspace_bytes, double* coef,
                        uint8_t* fit_status);
rs_status rs_predict_pooled(rs_ctx* ctx, const rs_batch* std, const double* coef,
                            const uint8_t* fit_status, int k, double tau, int flags,
                            uint32_t* rec_code, double* rec_pred, double* pred_all,
                            uint64_t* counters);

/* ---- A7: the plain predictor as the surrogate's fallback -----------------------------------
 * After rs_surrogate_infer has ranked one row per version of `batch` (raw counters, the
 * batch's row order) and set used_fallback[row] (device uint8 [n_rows]) where the row's
 * feature vector lies out of the training distribution, rs_surrogate_fallback predicts
 * those rows with the plain method instead: every program with at least one flagged row is
 * copied into a sub-batch in the workspace, the sub-batch goes through the whole plain pass
 * (rs_cv_step, FP64 Gram: standardization, Gram, fits, predictions, ranking; Sec. 2 tiers 2
 * and 3 with the Sec. 3.4 ridge model) over that program's splits in `splits` (the plain
 * protocol's train/test splits of every program of `batch`), and each flagged row takes the
 * plain ranking of its version from the first split of its program that tests it:
 * rec_code [n_rows] and rec_pred [n_rows][k] (device, the rs_predict_rank format, as
 * rs_surrogate_infer wrote them) are overwritten for those rows only; rows that no split
 * tests keep the surrogate's output.  Only the selected programs are standardized, Gram'd
 * and fitted.  refit (host int64 [2], nullable) receives the number of programs and of
 * versions that were refitted.  The call reads the selection's sizes back to the host
 * once (it synchronises the context's stream at that point), so it cannot be captured in a
 * CUDA graph.  workspace: rs_fallback_workspace_bytes(batch, splits) bytes (sized for every
 * program selected), 256-byte aligned, caller-owned; RS_ENOMEM if smaller.  lambda, k, tau
 * and flags (RS_RANK_ALL only) as in rs_cv_step.                                         */
size_t rs_fallback_workspace_bytes(const rs_batch* batch, const rs_splits* splits);
rs_status rs_surrogate_fallback(rs_ctx* ctx, const rs_batch* batch, const rs_splits* splits,
                                const uint8_t* used_fallback, double lambda, int k, double tau,
                                int flags, void* workspace, size_t workspace_bytes,
                                uint32_t* rec_code, double* rec_pred, int64_t* refit);

/* ---- A8: one graph launch per step, and the autotuner ---------------------------------------
 * rs_cv_graph_create runs rs_cv_step once eagerly (reporting argument errors), then captures
 * the same launch sequence into a CUDA graph bound to these pointers and sizes;
 * rs_cv_graph_launch replays it on the context's stream (one launch for the whole step,
 * ragged programs, versions and feature widths included).  Buffers must stay allocated
 * while the graph exists; their contents may change between launches.  Counters are added
 * to on every launch.  The graph uses the launch parameters the context holds at capture.
 * rs_autotune times the batched step on this batch for each candidate launch configuration
 * (the order in which the register solvers take their fits: 0 = largest first, 1 = ranges
 * alternately from the largest and the smallest end; the size at which fits move to the
 * register-heavier solver: 4..8; the rank pass's persistent grid: a quarter, half or all of
 * its resident blocks, given as 8, 16, 32), keeps the fastest in the context (used by every
 * later batched call), and writes the times (ms, at most *n_times: 30 candidates, order-major,
 * then size, then grid) if asked.  rs_get_tuning reports the context's current choice (any
 * pointer may be NULL); rs_set_tuning sets it (RS_EINVAL outside those values).  The
 * parameters change the work distribution only, never a result.                       */
typedef struct rs_graph rs_graph;
rs_status rs_cv_graph_create(rs_ctx* ctx, const rs_batch* batch, const rs_splits* splits,
                             double lambda, int k, double tau, int flags, int precision,
                             void* workspace, size_t workspace_bytes, int64_t* rec_offsets,
                             uint32_t* rec_code, double* rec_pred, double* pred_all,
                             uint64_t* counters, rs_graph** graph);
rs_status rs_cv_graph_launch(rs_graph* graph);
rs_status rs_cv_graph_destroy(rs_graph* graph);
rs_status rs_autotune(rs_ctx* ctx, const rs_batch* batch, const rs_splits* splits, double lambda,
                      int k, double tau, int flags, int precision, void* workspace,
                      size_t workspace_bytes, int64_t* rec_offsets, uint32_t* rec_code,
                      double* rec_pred, float* times_ms, int* n_times);
rs_status rs_get_tuning(const rs_ctx* ctx, int* solve_split, int* rank_waves, int* solve_order);
rs_status rs_set_tuning(rs_ctx* ctx, int solve_split, int rank_waves, int solve_order);
/* Tile shapes of the tensor-core Gram (RS_GRAM_BF16X3), chosen per feature width (rounded up
 * to a multiple of 64; a batch of mixed widths uses its widest): the output tile's width (32 or
 * 64 of the 64 columns of a program's block) and the split of its K = 3 x width contraction
 * (1: one CTA; 3: the three BF16 products hi hi^T, hi lo^T, lo hi^T on three CTAs, their FP32
 * results summed in FP64 in that order -- a result that can differ from the unsplit one in the
 * last FP32 bits).  rs_autotune_gram standardizes `batch` (raw counters) into the workspace
 * (at least rs_cv_workspace_bytes(batch, any splits) bytes) and times the Gram for the four
 * shapes, keeping the fastest in the context for that width; times_ms (host float [4],
 * nullable) gets the times in the order (64, 1), (32, 1), (64, 3), (32, 3), *choice (nullable)
 * the index kept.  rs_autotune does the same first when its precision is RS_GRAM_BF16X3.
 * rs_get_gram_tuning / rs_set_gram_tuning read or set the shape for a width.            */
rs_status rs_autotune_gram(rs_ctx* ctx, const rs_batch* batch, void* workspace, size_t workspace_bytes,
                           float* times_ms, int* choice);
rs_status rs_get_gram_tuning(const rs_ctx* ctx, int feat_width, int* tile_n, int* ksplit);
rs_status rs_set_gram_tuning(rs_ctx* ctx, int feat_width, int tile_n, int ksplit);

/* ---- tensor-core BF16 GEMM (the surrogate's and the tensor-core Gram's building block) ----
 * D[M][N] = A[M][K] * B[N][K]^T with A, B BF16 row-major (K contiguous, leading dimensions
 * lda, ldb in elements, multiples of 8, 16-byte aligned bases) and D FP32 row-major (ldd).
 * Runs on tcgen05 tensor cores (FP32 accumulation in tensor memory, TMA-fed shared memory
 * stages).  Not a step of the paper's method; exposed for tests and reuse.            */
rs_status rs_gemm_bf16(rs_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb,
                       float* D, int64_t ldd, int M, int N, int K);

/* ---- A7: the learned surrogate (not in the paper) -------------------------------------------
 * An MLP 256 -> 512 -> 512 -> 6 with GELU (tanh form: u (1 + tanh(sqrt(2/pi) (u + 0.044715
 * u^3))) / 2) maps a standardized feature vector to
 * the six predicted log speedups -- a learned stand-in for the tier-2 predictor (Sec. 2),
 * trained on labels that the plain ridge predictor produces.  BF16 weights and activations
 * on the tcgen05 tensor cores with FP32 accumulation, FP32 master weights, AdamW (beta1
 * 0.9, beta2 0.999, eps 1e-8), loss = mean squared error over the six outputs.
 * The state lives in one caller-owned FP32 "blob" of rs_surrogate_blob_bytes() bytes
 * (256-byte aligned).  rs_surrogate_offset(w) gives float offsets of: 0 W1 [512][256],
 * 1 b1 [512], 2 W2 [512][512], 3 b2 [512], 4 W3 [16][512] (rows 6..15 must be zero),
 * 5 b3 [16], 6 Adam m, 7 Adam v, 8 last gradients (each laid out like 0..5), 9 feature
 * mean [256] then std [256] of the training rows, 10 counters.  The caller writes the
 * initial weights and zeros the rest of the blob (m, v and the counters).
 * rs_surrogate_train: rows (double, [n][256] standardized features; labels [n][6] double,
 * NaN = no label, trained as 0) are taken in order in minibatches of cfg->batch_rows,
 * wrapping around; cfg->steps optimizer steps (0: only the feature statistics and the BF16
 * weight copies are prepared).  A call continues from the blob's counters: AdamW's step
 * count, and the minibatch position (wrapped into this call's rows).  use_graph = 1 captures one step in a CUDA graph and replays
 * it.  loss_curve (nullable, float [steps]) gets each minibatch's loss.
 * rs_surrogate_infer: X 16-byte aligned (RS_EINVAL otherwise; it is read with 16-byte
 * loads); pred [n][6] (float, nullable); ood_score [n] (nullable) = mean over
 * features of ((x - mean) / std)^2 against the training statistics; used_fallback [n]
 * (nullable) = 1 where ood_score > ood_threshold (those rows should be predicted by the
 * plain method).  With rec_code (nullable) the six outputs of each row are also ranked as
 * in rs_predict_rank (candidates: bits not set in masks[row]; all six with RS_RANK_ALL or
 * masks == NULL; threshold log(tau) compared in FP32; ties to the lower index; top k):
 * rec_code [n] and rec_pred [n][k] (double, nullable) in the rs_predict_rank format.
 * workspace: rs_surrogate_workspace_bytes(batch_rows) bytes, 256-byte aligned; inference
 * processes chunk_rows rows at a time (chunk_rows <= the batch_rows the workspace was
 * sized for).  RS_ETIMEOUT in the device status if a tensor-core pipeline wait gave up. */
typedef struct {
    int32_t batch_rows;
    int32_t use_graph;
    int64_t steps;
    float lr;
    float weight_decay;
} rs_mlp_cfg;
size_t rs_surrogate_blob_bytes(void);
int64_t rs_surrogate_offset(int which);
size_t rs_surrogate_workspace_bytes(int batch_rows);
rs_status rs_surrogate_train(rs_ctx* ctx, float* blob, const double* X, const double* Y, int64_t n,
                             const rs_mlp_cfg* cfg, float* loss_curve, void* workspace,
                             size_t workspace_bytes);
rs_status rs_surrogate_infer(rs_ctx* ctx, const float* blob, const double* X, int64_t n,
                             float ood_threshold, float* pred, float* ood_score,
                             uint8_t* used_fallback, const uint8_t* masks, int k, double tau,
                             int flags, uint32_t* rec_code, double* rec_pred, void* workspace,
                             size_t workspace_bytes, int chunk_rows);

/* ---- surrogate checkpoints ---------------------------------------------------------------
 * A checkpoint is a host byte buffer of rs_surrogate_checkpoint_bytes() bytes: a 64-byte
 * header (the magic "RSSURR01", format version 1, the layer widths 256, 512, 512 and 6, the
 * element type 0 = FP32, the optimizer steps taken so far (AdamW's t) and the blob's size in
 * bytes) followed by the whole blob: weights, Adam moments, last gradients, BF16 copies,
 * feature statistics and counters.  rs_surrogate_save copies the device blob into `host`
 * (host_bytes >= rs_surrogate_checkpoint_bytes(); ordered on the context's stream, and it
 * returns once the copy is complete).  rs_surrogate_restore checks the header (RS_EINVAL for a
 * wrong magic, version, width, type or size) and copies the blob back, returning once the
 * copy is complete.  rs_surrogate_train continues from the blob's counters, so s steps, a
 * save, a restore and t more steps on the same rows give the weights of s + t steps in one
 * run.  (The paper has no surrogate, so it has no checkpoint format either.)            */
size_t rs_surrogate_checkpoint_bytes(void);
rs_status rs_surrogate_save(rs_ctx* ctx, const float* blob, void* host, size_t host_bytes);
rs_status rs_surrogate_restore(rs_ctx* ctx, float* blob, const void* host, size_t host_bytes);

/* ---- the whole step, allocating nothing -------------------------------------------------
 * The paper has no counterpart: this is a deployment variant of rs_cv_step for callers that
 * cannot allocate device memory -- for instance a host that must finish all of its
 * cudaMalloc calls before it starts serving, or a caller that only owns the input and output
 * buffers it hands in and has no allocator to obtain a workspace from.  It runs the same
 * kernels as rs_cv_step (FP64 Gram, batched form) with its scratch (status words, the
 * row-planning scan, Z, the Gram blocks and the fit workspace) in one array of
 * RS_STATIC_SCRATCH_BYTES bytes that this library defines in device memory; every GPU that
 * loads the library keeps that array until the process exits.  It needs no rs_ctx and
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on a device (the current device) looks up the array's device address
 *     and caches it with the identity of the current CUDA context; make that first call
 *     before any stream capture.  If the context is destroyed and created again (after
 *     cudaDeviceReset, say) the next call looks the address up again, so it too should
 *     come before any capture.
 *   - Arguments follow rs_cv_step's rules (RS_EINVAL, with the reason in errbuf), and
 *     sizes that cannot fit are refused before any product of them is formed.
 *   - Every call uses the same array and leaves its contents behind; the call clears what
 *     must start at zero itself.  Calls whose work overlaps on the GPU (two streams, two
 *     threads) race on the array: serialise them.
 *   - A batch whose scratch would exceed RS_STATIC_SCRATCH_BYTES is rejected with
 *     RS_ENOMEM before anything is launched; errbuf (host, nullable) gets the reason.
 * Arguments as in rs_cv_step (X raw counters; the Gram is FP64; flags: RS_RANK_ALL only),
 * with the stream given directly.  rec_offsets (int64 [S+1]) is an output here.
 * device_status (device int, nullable) receives the device status word of the call
 * (0, or RS_EDATA / RS_ETIMEOUT as rs_check_device_status would report).              */
#define RS_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
rs_status rs_cv_step_static(void* cuda_stream, const rs_batch* batch, const rs_splits* splits,
                            double lambda, int k, double tau, int flags, int64_t* rec_offsets,
                            uint32_t* rec_code, double* rec_pred, double* pred_all,
                            uint64_t* counters, int* device_status, char* errbuf,
                            size_t errbuf_len);

#ifdef __cplusplus
}
#endif
#endif /* RS_H_ */
